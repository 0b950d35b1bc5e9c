"""Generalized advantage estimation and advantage normalisation (oracle, FP64).

Test infrastructure only.  GAE (Schulman et al., cited in Sec. 2.2.1) with gamma = 0.99 and
lambda = 0.95 (Table 3), written as the reverse-time recursion over the n_steps of each
robot (Sec. 2.2.1: B = n_robots * n_steps), with episode ends cutting the recursion:

    delta_t = r_t + gamma (1 - d_t) V_{t+1} - V_t
    A_t     = delta_t + gamma lambda (1 - d_t) A_{t+1},      A_T = 0, V_T = critic(o_T)
    R_t     = A_t + V_t                                        (critic target)

Time-out bootstrapping (Sec. 2.2.2) is already folded into r_t by the env step.
Normalisation over the whole batch (population std, + 1e-8) is the usual PPO practice;
the paper is silent on it.
"""
import numpy as np


def gae(rew, val, last_val, done, gamma, lam):
    """rew, val: [T, N]; last_val: [N]; done: [T, N] (0/1).  Returns (A, R) [T, N] float64."""
    rew = np.asarray(rew, np.float64)
    val = np.asarray(val, np.float64)
    done = np.asarray(done, np.float64)
    T, N = rew.shape
    A = np.zeros((T, N))
    next_a = np.zeros(N)
    next_v = np.asarray(last_val, np.float64)
    for t in range(T - 1, -1, -1):
        nonterm = 1.0 - done[t]
        delta = rew[t] + gamma * nonterm * next_v - val[t]
        next_a = delta + gamma * lam * nonterm * next_a
        A[t] = next_a
        next_v = val[t]
    return A, A + val


def normalize(adv, eps=1e-8):
    """(A - mean) / (std + eps) over the whole batch; population standard deviation."""
    adv = np.asarray(adv, np.float64)
    m = adv.mean()
    s = np.sqrt(((adv - m) ** 2).mean())
    return (adv - m) / (s + eps), m, s
