"""Shared test helpers: one set of workload numbers turned into the library's config and the
oracle's configs, tolerances, and norm-wise error measures."""
import numpy as np

from oracle import config as OC

# Tolerances (relative, norm-wise per tensor: |x - ref|_inf / max(|ref|_inf, 1e-30)).
TOL_FP32 = 1e-5
TOL_BF16 = 2e-2


def rel_err(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.abs(x - ref).max() / max(np.abs(ref).max(), 1e-30)) if ref.size else 0.0


def workload(name, **over):
    """Named synthetic workloads (numbers shared by the library config and the oracle)."""
    w = dict(num_envs=64, num_steps=24, grid=(17, 11), hidden=(64, 64), epochs=1, minibatches=2,
             precision=0, seed=0, noise_on=1, push_on=1, crash_threshold=9170000)
    if name == "tiny":          # 64 envs x 24, obs 48, 64-64 (plain PPO iteration)
        w.update(grid=(0, 0))
    elif name == "flat":        # 4096 x 24, obs 48, 512-256-128, FP32
        w.update(num_envs=4096, grid=(0, 0), hidden=(512, 256, 128), epochs=5, minibatches=4)
    elif name == "rough":       # 4096 x 24, obs 235, 512-256-128
        w.update(num_envs=4096, hidden=(512, 256, 128), epochs=5, minibatches=4)
    elif name == "small_rough":
        w.update(num_envs=320, num_steps=8, hidden=(128, 128), epochs=1, minibatches=1)
    else:
        raise KeyError(name)
    w.update(over)
    return w


def lib_config(w):
    from paper_2109_11978_b300 import api
    gx, gy = w["grid"]
    O = 48 + gx * gy
    Op = (O + 63) // 64 * 64
    return api.default_config(
        num_envs=w["num_envs"], num_steps=w["num_steps"], grid_x=gx, grid_y=gy, obs_dim=O, obs_pad=Op,
        hidden=list(w["hidden"]), epochs=w["epochs"], minibatches=w["minibatches"], precision=w["precision"],
        seed=w["seed"], noise_on=w["noise_on"], push_on=w["push_on"], crash_threshold=w["crash_threshold"])


def oracle_env_config(w):
    gx, gy = w["grid"]
    return OC.EnvConfig(num_envs=w["num_envs"], grid_x=gx, grid_y=gy, seed=w["seed"], noise_on=bool(w["noise_on"]),
                        push_on=bool(w["push_on"]), crash_threshold=w["crash_threshold"])


def oracle_ppo_config(w):
    return OC.PPOConfig(epochs=w["epochs"], minibatches=w["minibatches"], seed=w["seed"])


def obs_dims(w):
    gx, gy = w["grid"]
    O = 48 + gx * gy
    return O, (O + 63) // 64 * 64
