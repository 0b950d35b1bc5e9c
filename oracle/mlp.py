"""Actor and critic MLPs, Gaussian policy head (oracle, FP64).

Test infrastructure only.  The paper's policy and critic are neural networks evaluated on
the GPU for every robot (Sec. 2, App. A.1); the architecture (ELU hidden layers of
512-256-128, linear heads, a state-independent learned log standard deviation per action)
is the configuration this build is measured on.  The Gaussian policy's sampling, log
density and entropy are the textbook diagonal-Gaussian forms used by PPO (Sec. 2.2).

Flat parameter layout (also the library's): actor [W1, b1, ..., W_L+1, b_L+1, log_std]
then critic [W1, b1, ..., W_L+1, b_L+1]; W_l is [fan_out, fan_in] row-major; the first layer's
fan_in is the logical observation size (no padding).
"""
import numpy as np

from . import rng

LOG_2PI = np.log(2.0 * np.pi)


def elu(x):
    return np.where(x > 0, x, np.expm1(np.minimum(x, 0.0)))


def elu_grad_from_output(y):
    """d ELU / dx expressed through y = ELU(x): 1 for x > 0, exp(x) = y + 1 otherwise."""
    return np.where(y > 0, 1.0, y + 1.0)


def layer_dims(obs_dim, hidden, out_dim):
    dims = [obs_dim] + list(hidden) + [out_dim]
    return list(zip(dims[1:], dims[:-1]))          # (fan_out, fan_in) per layer


def param_count(obs_dim, hidden, act_dim):
    a = sum(o * i + o for o, i in layer_dims(obs_dim, hidden, act_dim)) + act_dim
    c = sum(o * i + o for o, i in layer_dims(obs_dim, hidden, 1))
    return a + c


def unflatten(flat, obs_dim, hidden, act_dim):
    flat = np.asarray(flat, np.float64)
    p, off = {"actor": [], "critic": []}, 0
    for net, out in (("actor", act_dim), ("critic", 1)):
        for o, i in layer_dims(obs_dim, hidden, out):
            W = flat[off:off + o * i].reshape(o, i)
            off += o * i
            b = flat[off:off + o]
            off += o
            p[net].append((W, b))
        if net == "actor":
            p["log_std"] = flat[off:off + act_dim]
            off += act_dim
    assert off == flat.size, (off, flat.size)
    return p


def flatten(p):
    parts = []
    for W, b in p["actor"]:
        parts += [W.ravel(), b.ravel()]
    parts.append(p["log_std"].ravel())
    for W, b in p["critic"]:
        parts += [W.ravel(), b.ravel()]
    return np.concatenate(parts)


def forward(layers, x):
    """Returns (output, [x, h_1, ..., h_L]) with ELU hidden layers and a linear head."""
    hs = [np.asarray(x, np.float64)]
    for l, (W, b) in enumerate(layers):
        z = hs[-1] @ W.T + b
        if l < len(layers) - 1:
            hs.append(elu(z))
        else:
            return z, hs
    raise AssertionError


def log_prob(a, mu, log_std):
    """log N(a; mu, diag(exp(log_std))^2), summed over action dimensions."""
    var = np.exp(2.0 * log_std)
    return (-(a - mu) ** 2 / (2.0 * var) - log_std - 0.5 * LOG_2PI).sum(-1)


def entropy(log_std):
    """Entropy of the diagonal Gaussian: sum_j (log sigma_j + 0.5 log(2 pi e))."""
    return float((log_std + 0.5 * (LOG_2PI + 1.0)).sum())


def kl_old_new(mu_old, log_std_old, mu_new, log_std_new):
    """KL(pi_old || pi_new) per sample, summed over action dimensions (closed form)."""
    so2 = np.exp(2.0 * log_std_old)
    sn2 = np.exp(2.0 * log_std_new)
    return (log_std_new - log_std_old + (so2 + (mu_old - mu_new) ** 2) / (2.0 * sn2) - 0.5).sum(-1)


def act(params, obs, seed, iteration, t, env=None):
    """Policy inference for one step: a = mu + sigma * eps, log pi(a), mu, V (Sec. 2.2).

    eps_j is the Box-Muller normal of word j of the act-stream key of (iteration, t, env).
    """
    obs = np.asarray(obs, np.float64)
    n = obs.shape[0]
    env = np.arange(n) if env is None else env
    mu, _ = forward(params["actor"], obs)
    v, _ = forward(params["critic"], obs)
    key = rng.key(seed, rng.STREAM_ACT, iteration, t, env)
    eps = np.stack([rng.box_muller_f64(rng.word(key, j)) for j in range(mu.shape[1])], 1)
    sigma = np.exp(params["log_std"])
    a = mu + sigma * eps
    return {"actions": a, "mu": mu, "logp": log_prob(a, mu, params["log_std"]),
            "values": v[:, 0], "eps": eps}
