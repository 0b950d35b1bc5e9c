"""One full training iteration: rollout of n_steps for all robots, GAE, PPO update (oracle).

Test infrastructure only.  The iteration of Sec. 2 / Sec. 2.2: with a fixed policy, every
robot takes n_steps policy steps (inference, env math, storage), then the critic values the
final observation, advantages are estimated and the policy is updated for the Table 3
epochs x minibatches.  The random key of step t of iteration i is (seed, stream, i, t, env).
"""
import numpy as np

from . import env as envmod
from . import gae as gaemod
from . import mlp, ppo


class Learner:
    """Oracle state of one learner: env state, observation, parameters, Adam, alpha."""

    def __init__(self, ecfg, pcfg, hidden, hf, flat_params, sf=None, si=None, obs=None):
        self.ecfg, self.pcfg, self.hidden, self.hf = ecfg, pcfg, tuple(hidden), hf
        self.flat = np.asarray(flat_params, np.float64).copy()
        self.adam = ppo.Adam(self.flat.size)
        self.lr = pcfg.lr_init
        self.iteration = 0
        if sf is None:
            sf, si = envmod.initial_state(ecfg)
            obs = initial_observation(ecfg, hf, sf, si)
        self.sf, self.si, self.obs = sf.copy(), si.copy(), np.asarray(obs, np.float64).copy()

    def params(self):
        return mlp.unflatten(self.flat, self.ecfg.obs_dim, self.hidden, self.ecfg.act_dim)

    def rollout(self, T, actions_override=None, values_override=None):
        """T policy steps.  actions_override[t] (if given) replaces the sampled actions, so
        the env math can be driven by another implementation's actions (teacher forcing);
        values_override[t] likewise replaces V(o_t) where the env step uses it (the time-out
        bootstrap of Sec. 2.2.2 adds gamma V(o_t), the value stored at act time).  The oracle's
        own sampled actions and values are kept under "sampled_actions" and "values"."""
        N, O, A = self.ecfg.num_envs, self.ecfg.obs_dim, self.ecfg.act_dim
        st = {"obs": np.zeros((T, N, O)), "actions": np.zeros((T, N, A)), "mu": np.zeros((T, N, A)),
              "sampled_actions": np.zeros((T, N, A)),
              "logp": np.zeros((T, N)), "values": np.zeros((T, N)), "reward": np.zeros((T, N)),
              "done": np.zeros((T, N), np.uint8), "timeout": np.zeros((T, N), np.uint8),
              "level": np.zeros((T, N), np.int32)}
        p = self.params()
        for t in range(T):
            out = mlp.act(p, self.obs, self.ecfg.seed, self.iteration, t)
            a = out["actions"] if actions_override is None else np.asarray(actions_override[t], np.float64)
            v = out["values"] if values_override is None else np.asarray(values_override[t], np.float64)
            st["obs"][t] = self.obs
            st["actions"][t], st["mu"][t] = a, out["mu"]
            st["sampled_actions"][t] = out["actions"]
            st["logp"][t] = mlp.log_prob(a, out["mu"], p["log_std"])
            st["values"][t] = out["values"]
            r = envmod.step(self.ecfg, self.hf, self.sf, self.si, a.astype(np.float32),
                            v, self.iteration, t)
            self.sf, self.si, self.obs = r["sf"], r["si"], r["obs"]
            st["reward"][t], st["done"][t], st["timeout"][t] = r["reward"], r["done"], r["timeout"]
            st["level"][t] = r["level"]
        st["last_values"] = mlp.forward(p["critic"], self.obs)[0][:, 0]
        return st

    def iterate(self, T):
        st = self.rollout(T)
        A, R = gaemod.gae(st["reward"], st["values"], st["last_values"], st["done"],
                          self.pcfg.gamma, self.pcfg.lam)
        An, _, _ = gaemod.normalize(A)
        B = T * self.ecfg.num_envs
        batch = {"obs": st["obs"].reshape(B, -1), "actions": st["actions"].reshape(B, -1),
                 "logp": st["logp"].reshape(B), "mu": st["mu"].reshape(B, -1),
                 "values": st["values"].reshape(B), "adv": An.reshape(B), "ret": R.reshape(B)}
        self.flat, self.lr, stats = ppo.update(self.flat, self.adam, self.lr, batch,
                                               self.ecfg.obs_dim, self.hidden, self.ecfg.act_dim,
                                               self.pcfg, self.iteration)
        self.iteration += 1
        return st, stats


def initial_observation(ecfg, hf, sf, si):
    """Observation of the freshly spawned robots; noise drawn from the init-stream key."""
    from . import rng
    env = np.arange(sf.shape[1])
    key = rng.key(ecfg.seed, rng.STREAM_INIT, 0, 0, env)
    return envmod.observe(ecfg, hf, envmod.unpack(sf, si), env, key)
