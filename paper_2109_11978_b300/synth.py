"""Seeded synthetic inputs (terrain, initial weights, env states, rollout batches).

This module only draws inputs: it holds none of the method's arithmetic and is the one
module that both the CUDA path's callers (tests, bench, smoke) and the oracle's callers use.
Every generator is numpy with an explicit seed.  The shapes follow the workloads of the
paper (4096 robots x 24 steps, 12 actions, 8 m terrain tiles at 0.1 m, 10 levels x 20
terrain columns, 17 x 11 height samples) and the configurations this build is measured on.
"""
import numpy as np

# Row layout of the fp32 SoA env state [57, N] and the int32 state [3, N].
F_PX, F_PY, F_Z, F_HC, F_HS = 0, 1, 2, 3, 4
F_VX, F_VY, F_VZ, F_WX, F_WY, F_WZ = 5, 6, 7, 8, 9, 10
F_GX, F_GY, F_GZ = 11, 12, 13
F_CMDX, F_CMDY, F_CMDW = 14, 15, 16
F_TAIR, F_Q, F_QD, F_AP = 17, 21, 33, 45
NF, NI = 57, 3
I_EPLEN, I_LEVEL, I_CONTACT = 0, 1, 2


def heightfield(seed, num_levels=10, num_cols=20, cells_per_tile=80, max_height=0.2, flat=False):
    """Rough-terrain heightfield [num_levels * c, num_cols * c] fp32 (x rows, y columns).

    Each cell of a tile on level l is uniform in [0, max_height * l / (num_levels - 1)], so the
    first row of tiles is flat and difficulty grows with the level (Sec. 3.1 curriculum).
    """
    nx, ny = num_levels * cells_per_tile, num_cols * cells_per_tile
    if flat:
        return np.zeros((nx, ny), np.float32)
    rs = np.random.default_rng(seed)
    u = rs.random((nx, ny))
    level = np.arange(nx) // cells_per_tile
    scale = max_height * level / max(num_levels - 1, 1)
    return (u * scale[:, None]).astype(np.float32)


def affine_heightfield(shape, a, b, c):
    """H[i, j] = a * x_i + b * y_j + c at grid spacing 1 (caller scales); fp32."""
    i = np.arange(shape[0])[:, None]
    j = np.arange(shape[1])[None, :]
    return (a * i + b * j + c).astype(np.float32)


def layer_dims(obs_dim, hidden, out_dim):
    dims = [obs_dim] + list(hidden) + [out_dim]
    return list(zip(dims[1:], dims[:-1]))


def xavier_params(seed, obs_dim, hidden, act_dim, log_std=0.0, bias_scale=0.0):
    """Flat fp32 parameters: Xavier-uniform weights, biases (0 unless bias_scale), log_std.

    Layout: actor [W1, b1, ..., W_head, b_head, log_std], critic [W1, b1, ..., W_head, b_head];
    W is [fan_out, fan_in] row-major.
    """
    rs = np.random.default_rng(seed)
    parts = []
    for out in (act_dim, 1):
        for o, i in layer_dims(obs_dim, hidden, out):
            lim = np.sqrt(6.0 / (i + o))
            parts.append(rs.uniform(-lim, lim, o * i))
            parts.append(rs.uniform(-bias_scale, bias_scale, o) if bias_scale else np.zeros(o))
        if out == act_dim:
            parts.append(np.full(act_dim, log_std))
    return np.concatenate(parts).astype(np.float32)


def random_env_state(seed, num_envs, num_levels=10, max_episode_len=1000, radius=6.0,
                     near_timeout_frac=0.1):
    """A diverse fp32/int32 env state: positions inside and outside the 4 m promotion radius,
    all levels, episode lengths spread over [0, max) with a share one step from the time-out,
    random commands, unit headings, joint states and previous actions."""
    rs = np.random.default_rng(seed)
    n = num_envs
    sf = np.zeros((NF, n), np.float32)
    r = radius * np.sqrt(rs.random(n))
    th = rs.uniform(-np.pi, np.pi, n)
    sf[F_PX], sf[F_PY] = r * np.cos(th), r * np.sin(th)
    sf[F_Z] = 0.5 + 0.0625 * rs.integers(0, num_levels, n) + rs.normal(0, 0.01, n)
    yaw = rs.uniform(-np.pi, np.pi, n)
    sf[F_HC], sf[F_HS] = np.cos(yaw), np.sin(yaw)
    sf[F_VX:F_VZ + 1] = rs.normal(0, 0.5, (3, n))
    sf[F_WX:F_WZ + 1] = rs.normal(0, 0.3, (3, n))
    g = rs.normal(0, 0.05, (2, n))
    sf[F_GX], sf[F_GY] = g
    sf[F_GZ] = -np.sqrt(1 - (g ** 2).sum(0))
    sf[F_CMDX:F_CMDW + 1] = rs.uniform(-1, 1, (3, n))
    sf[F_TAIR:F_TAIR + 4] = rs.integers(0, 30, (4, n)) * np.float32(0.02)
    sf[F_Q:F_Q + 12] = rs.normal(0, 0.3, (12, n))
    sf[F_QD:F_QD + 12] = rs.normal(0, 1.0, (12, n))
    sf[F_AP:F_AP + 12] = rs.normal(0, 1.0, (12, n))
    si = np.zeros((NI, n), np.int32)
    ep = rs.integers(0, max_episode_len, n)
    near = rs.random(n) < near_timeout_frac
    ep[near] = max_episode_len - 1
    si[I_EPLEN] = ep
    si[I_LEVEL] = rs.integers(0, num_levels, n)
    si[I_CONTACT] = rs.integers(0, 16, n)
    return sf, si


def gaussian_rollout(seed, T, N, obs_dim, act_dim, reset_prob=0.05, rho=0.9):
    """Synthetic rollout for the learner: obs from a seeded linear-Gaussian transition
    (o_{t+1} = rho o_t + sqrt(1 - rho^2) xi, marginally N(0, 1)), rewards N(0, 1), ~5 %
    random resets (done and time-out flags), actions near a random policy."""
    rs = np.random.default_rng(seed)
    obs = np.zeros((T, N, obs_dim), np.float32)
    o = rs.standard_normal((N, obs_dim))
    for t in range(T):
        obs[t] = o
        o = rho * o + np.sqrt(1 - rho * rho) * rs.standard_normal((N, obs_dim))
    return {
        "obs": obs,
        "last_obs": o.astype(np.float32),
        "rewards": rs.standard_normal((T, N)).astype(np.float32),
        "dones": (rs.random((T, N)) < reset_prob).astype(np.uint8),
        "eps": rs.standard_normal((T, N, act_dim)).astype(np.float32),
    }
