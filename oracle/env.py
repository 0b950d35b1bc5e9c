"""Env-side tensor math of one 50 Hz policy step for N robots (oracle, FP64).

Test infrastructure only.  Follows the paper:
* actions are joint-position targets tracked by a PD controller (Sec. 3.2); 4 simulation
  substeps of 0.005 s per 0.02 s policy step (App. A.1.1), the PD torque recomputed every
  substep.  q* = q_def + action_scale * a (the paper only says "desired joint positions").
* reward = sum of the nine Table 2 terms, each weight times dt (App. A.3, Table 2);
* base contact = crash = reset; time-out after the 20 s maximum episode length
  (Sec. 2.2.1, Sec. 3.2); the time-out reward is bootstrapped with gamma * V (Sec. 2.2.2);
* game-inspired curriculum at reset (Sec. 3.1): promote past the tile border, demote if the
  robot covered less than half the commanded distance, loop back to a random level past
  the top; robots move to the centre of their new tile (Sec. 2.1 tiled terrain);
* commands resampled at reset and held for the episode (Sec. 3.1);
* observation = [v_b, w_b, g, commands, q - q_def, qd, previous actions, terrain heights]
  (Sec. 3.2) plus uniform noise with the Table 4 half-widths (Sec. 3.3, App. A.5);
  heights = base height minus terrain height at grid points around the base (Sec. 3.2),
  read bilinearly from the heightfield;
* pushes every 10 s of up to +-1 m/s in x and y (Sec. 3.3).

The stand-in physics (oracle.standin) is the only fp32 part; everything the method computes
from its output (reward, observation, decisions) is float64 here.  Integer decisions that
depend on floats (curriculum distances) are taken in float64 from the stand-in's fp32
state with one rounding per operation, in the order written below.
"""
import numpy as np

from . import config as C
from . import rng, standin

f32 = np.float32

# Row layout of the fp32 SoA state matrix [NF, N] (same meaning as the library's layout).
F_PX, F_PY, F_Z, F_HC, F_HS = 0, 1, 2, 3, 4
F_VX, F_VY, F_VZ, F_WX, F_WY, F_WZ = 5, 6, 7, 8, 9, 10
F_GX, F_GY, F_GZ = 11, 12, 13
F_CMDX, F_CMDY, F_CMDW = 14, 15, 16
F_TAIR = 17          # 4 rows
F_Q = 21             # 12 rows
F_QD = 33            # 12 rows
F_AP = 45            # 12 rows (previous actions)
NF = 57
I_EPLEN, I_LEVEL, I_CONTACT = 0, 1, 2
NI = 3

_SCALARS = {"px": F_PX, "py": F_PY, "z": F_Z, "hc": F_HC, "hs": F_HS, "vx": F_VX, "vy": F_VY,
            "vz": F_VZ, "wx": F_WX, "wy": F_WY, "wz": F_WZ, "gx": F_GX, "gy": F_GY, "gz": F_GZ,
            "cmdx": F_CMDX, "cmdy": F_CMDY, "cmdw": F_CMDW}
_VECTORS = {"tair": (F_TAIR, 4), "q": (F_Q, 12), "qd": (F_QD, 12), "ap": (F_AP, 12)}


def unpack(sf, si):
    S = {k: sf[r].astype(f32).copy() for k, r in _SCALARS.items()}
    for k, (r, n) in _VECTORS.items():
        S[k] = sf[r:r + n].astype(f32).copy()
    S["eplen"] = si[I_EPLEN].astype(np.int64).copy()
    S["level"] = si[I_LEVEL].astype(np.int64).copy()
    S["contact"] = si[I_CONTACT].astype(np.int64).copy()
    return S


def pack(S):
    n = S["px"].shape[0]
    sf = np.zeros((NF, n), f32)
    for k, r in _SCALARS.items():
        sf[r] = S[k]
    for k, (r, m) in _VECTORS.items():
        sf[r:r + m] = S[k]
    si = np.zeros((NI, n), np.int32)
    si[I_EPLEN] = S["eplen"]
    si[I_LEVEL] = S["level"]
    si[I_CONTACT] = S["contact"]
    return sf, si


def bilinear(hf, x, y, res):
    """Terrain height at world (x, y) (float64), bilinear on the grid, clamped at the border."""
    nx, ny = hf.shape
    u = np.clip(x / res, 0.0, nx - 1.0)
    v = np.clip(y / res, 0.0, ny - 1.0)
    i0 = np.minimum(np.floor(u).astype(np.int64), nx - 2)
    j0 = np.minimum(np.floor(v).astype(np.int64), ny - 2)
    fu = u - i0
    fv = v - j0
    h = hf.astype(np.float64)
    return ((1 - fu) * (1 - fv) * h[i0, j0] + fu * (1 - fv) * h[i0 + 1, j0]
            + (1 - fu) * fv * h[i0, j0 + 1] + fu * fv * h[i0 + 1, j0 + 1])


def grid_offsets(cfg):
    """Body-frame (x, y) offsets of the height samples; sample index k = iy * grid_x + ix."""
    ix = np.arange(cfg.grid_x) - (cfg.grid_x - 1) / 2.0
    iy = np.arange(cfg.grid_y) - (cfg.grid_y - 1) / 2.0
    gx = np.tile(ix, cfg.grid_y) * cfg.grid_spacing
    gy = np.repeat(iy, cfg.grid_x) * cfg.grid_spacing
    return gx, gy



def pd_torque(q_target, q, qd, kp, kd):
    """PD controller of Sec. 3.2: tau = Kp (q* - q) - Kd qd (float64)."""
    return kp * (np.asarray(q_target, np.float64) - np.asarray(q, np.float64)) - kd * np.asarray(qd, np.float64)


def reward_terms(v, w, cmd, qd, qd_prev, tau, a, a_prev, n_coll, tair, first, dt):
    """The nine weighted Table 2 terms (before the common factor dt), float64.

    v, w: base linear / angular velocity components; cmd = (v*_x, v*_y, w*_z); qd, qd_prev:
    joint velocities now and one policy step ago ([12, N]); joint acceleration
    qdd = (qd - qd_prev) / dt; tau: torque of the last substep; a, a_prev: actions now and at
    the previous step (the action rate |a_t - a_{t-1}|^2); n_coll: collision count; tair:
    feet air times; first: 1 on the step a foot touches down (the air-time term counts then).
    """
    phi = lambda sq: np.exp(-sq / C.PHI_SCALE)
    vx, vy, vz = v
    wx, wy, wz = w
    cx, cy, cw = cmd
    qdd = (qd - qd_prev) / dt
    return np.stack([
        C.W_LIN_VEL * phi((cx - vx) ** 2 + (cy - vy) ** 2),
        C.W_ANG_VEL * phi((cw - wz) ** 2),
        C.W_VZ * -(vz ** 2),
        C.W_WXY * -(wx ** 2 + wy ** 2),
        C.W_JOINT * -((qdd ** 2).sum(0) + (qd ** 2).sum(0)),
        C.W_TORQUE * -(tau ** 2).sum(0),
        C.W_ACTION_RATE * -((a - a_prev) ** 2).sum(0),
        C.W_COLLISION * -np.asarray(n_coll, np.float64),
        C.W_AIR_TIME * ((tair - C.AIR_TIME_TARGET) * first).sum(0),
    ])


def termination(eplen_new, crash, max_episode_len):
    """Crash (base contact) or time-out after the maximum episode length (Sec. 2.2.1, 3.2).
    A crash on the last step counts as a crash, not as a time-out."""
    timeout = (np.asarray(eplen_new) >= max_episode_len) & ~np.asarray(crash, bool)
    return np.asarray(crash, bool) | timeout, timeout


def bootstrap_timeout(reward, values, timeout, gamma):
    """Sec. 2.2.2: on a time-out the critic target is bootstrapped with its own prediction,
    r <- r + gamma V(o_t)."""
    return np.asarray(reward, np.float64) + gamma * np.asarray(values, np.float64) * np.asarray(timeout)


def curriculum_predicates(cfg, px, py, cmdx, cmdy):
    """Promotion / demotion tests of Sec. 3.1 in float64 from fp32 inputs.

    promote: the robot walked past the border of its 8 m tile, |p - origin| > tile / 2;
    demote:  it covered less than half the distance its command asked for over the maximum
             episode duration, |p - origin| < 0.5 |v*_xy| T_max.  Squared distances, one
             rounding per operation in this order.
    """
    px, py = np.asarray(px, np.float64), np.asarray(py, np.float64)
    cx, cy = np.asarray(cmdx, np.float64), np.asarray(cmdy, np.float64)
    d2 = px * px + py * py
    half = 0.5 * np.float64(f32(cfg.tile_size))
    promote = d2 > half * half
    vv = cx * cx + cy * cy
    T = np.float64(cfg.max_episode_len) * np.float64(f32(cfg.dt))
    thr = (vv * (T * T)) * 0.25
    return promote, d2 < thr, d2, thr


def curriculum_level(level, promote, demote, loop_level, num_levels):
    """Level at the next reset (Sec. 3.1): promotion wins over demotion; demotion stops at 0;
    a promotion from the top level loops back to a random level (loop_level)."""
    level = np.asarray(level)
    up = np.where(level + 1 >= num_levels, loop_level, level + 1)
    return np.where(promote, up, np.where(demote, np.maximum(level - 1, 0), level))


def spawn_origin(cfg, level, env):
    """Centre of the robot's tile: level selects the row (x), env mod num_cols the column (y)."""
    col = env % cfg.num_cols
    return (level + 0.5) * cfg.tile_size, (col + 0.5) * cfg.tile_size


def observe(cfg, hf, S, env, key):
    """Observation rows [N, obs_dim] in float64 from the (post-reset) fp32 state (Sec. 3.2)."""
    n = env.shape[0]
    o = np.zeros((n, cfg.obs_dim))
    d = lambda a: np.asarray(a, np.float64)
    o[:, 0], o[:, 1], o[:, 2] = d(S["vx"]), d(S["vy"]), d(S["vz"])
    o[:, 3], o[:, 4], o[:, 5] = d(S["wx"]), d(S["wy"]), d(S["wz"])
    o[:, 6], o[:, 7], o[:, 8] = d(S["gx"]), d(S["gy"]), d(S["gz"])
    o[:, 9], o[:, 10], o[:, 11] = d(S["cmdx"]), d(S["cmdy"]), d(S["cmdw"])
    o[:, 12:24] = (d(S["q"]) - d(cfg.q_def)[:, None]).T
    o[:, 24:36] = d(S["qd"]).T
    o[:, 36:48] = d(S["ap"]).T
    if cfg.num_heights:
        ox, oy = spawn_origin(cfg, S["level"].astype(np.float64), env)
        bx = ox + d(S["px"])
        by = oy + d(S["py"])
        c, s = d(S["hc"]), d(S["hs"])
        gx, gy = grid_offsets(cfg)
        X = bx[:, None] + c[:, None] * gx[None, :] - s[:, None] * gy[None, :]
        Y = by[:, None] + s[:, None] * gx[None, :] + c[:, None] * gy[None, :]
        o[:, 48:] = d(S["z"])[:, None] - bilinear(hf, X, Y, cfg.hf_res)
    if cfg.noise_on:
        scales = cfg.noise_scales()
        for k in range(cfg.obs_dim):
            w = rng.word(key, C.SLOT_OBS_NOISE + k // 2)
            u32 = rng.hi32(w) if k % 2 == 0 else rng.lo32(w)
            o[:, k] += scales[k] * rng.uniform_pm1_f32(u32).astype(np.float64)
    return o


def reset_state(cfg, S, mask, key, level_new):
    """Respawn masked robots at the centre of their tile with fresh commands (Sec. 3.1)."""
    m = mask
    S["level"] = np.where(m, level_new, S["level"])
    S["px"][m] = 0
    S["py"][m] = 0
    S["z"] = np.where(m, standin.z_nominal(S["level"]), S["z"]).astype(f32)
    hx = rng.uniform_pm1_f32(rng.hi32(rng.word(key, C.SLOT_HEADING)))
    hy = rng.uniform_pm1_f32(rng.hi32(rng.word(key, C.SLOT_HEADING + 1)))
    n2 = hx * hx + hy * hy
    ok = n2 > f32(2.0 ** -20)
    nn = np.sqrt(np.where(ok, n2, f32(1.0)))
    hc = np.where(ok, hx / nn, f32(1.0)).astype(f32)
    hs = np.where(ok, hy / nn, f32(0.0)).astype(f32)
    S["hc"] = np.where(m, hc, S["hc"]).astype(f32)
    S["hs"] = np.where(m, hs, S["hs"]).astype(f32)
    for name in ("vx", "vy", "vz", "wx", "wy", "wz", "gx", "gy"):
        S[name][m] = 0
    S["gz"][m] = -1
    for i, name in enumerate(("cmdx", "cmdy", "cmdw")):
        u = rng.uniform_pm1_f32(rng.hi32(rng.word(key, C.SLOT_CMD + i)))
        S[name] = np.where(m, (u * f32(cfg.cmd_range[i])).astype(f32), S[name]).astype(f32)
    S["tair"][:, m] = 0
    S["q"][:, m] = cfg.q_def.astype(f32)[:, None]
    S["qd"][:, m] = 0
    S["ap"][:, m] = 0
    S["eplen"][m] = 0
    S["contact"][m] = 0


def initial_state(cfg, randomize_eplen=True):
    """All robots spawned on level 0 (Sec. 3.1: training starts on the first row)."""
    n = cfg.num_envs
    env = np.arange(n)
    S = {k: np.zeros(n, f32) for k in _SCALARS}
    S["hc"][:] = 1
    S["gz"][:] = -1
    S["tair"] = np.zeros((4, n), f32)
    S["q"] = np.repeat(cfg.q_def.astype(f32)[:, None], n, axis=1)
    S["qd"] = np.zeros((12, n), f32)
    S["ap"] = np.zeros((12, n), f32)
    S["eplen"] = np.zeros(n, np.int64)
    S["level"] = np.zeros(n, np.int64)
    S["contact"] = np.zeros(n, np.int64)
    key = rng.key(cfg.seed, rng.STREAM_INIT, 0, 0, env)
    reset_state(cfg, S, np.ones(n, bool), key, np.zeros(n, np.int64))
    if randomize_eplen:
        S["eplen"] = rng.mulhi32(rng.hi32(rng.word(key, C.SLOT_EPLEN)), cfg.max_episode_len)
    return pack(S)


def contact_schedule(env, eplen):
    """Foot contact bits of the stand-in after a step: integer trot-like schedule."""
    bits = np.zeros_like(eplen)
    off = (env * C.CONTACT_ENV_STRIDE) % C.CONTACT_PERIOD
    for f in range(4):
        on = ((eplen + off + C.CONTACT_PHASE[f]) % C.CONTACT_PERIOD) < C.CONTACT_DUTY
        bits |= on.astype(np.int64) << f
    return bits


def step(cfg, hf, sf, si, actions, values, iteration, t):
    """One policy step for all robots.

    Inputs: fp32 state (sf [NF, N], si [NI, N]), actions [N, 12], values V(o_t) [N] (for the
    time-out bootstrap), counters (iteration, t) of the random key.
    Returns dict: state (sf, si), obs [N, obs_dim] f64, reward [N] f64, done, timeout (u8),
    level, terrain_idx (int32), plus diagnostics (tau of the last substep, pre-reset position).
    """
    n = sf.shape[1]
    env = np.arange(n)
    S = unpack(sf, si)
    key = rng.key(cfg.seed, rng.STREAM_ENV, iteration, t, env)
    a32 = np.asarray(actions, f32).T.copy()            # [12, N]
    a64 = a32.astype(np.float64)
    qd_old64 = S["qd"].astype(np.float64)
    ap64 = S["ap"].astype(np.float64)

    # Pushes (Sec. 3.3): every push_interval steps of the episode, on the velocity state.
    if cfg.push_on:
        pm = (S["eplen"] > 0) & (S["eplen"] % cfg.push_interval == 0)
        ux = rng.uniform_pm1_f32(rng.hi32(rng.word(key, C.SLOT_PUSH_X)))
        uy = rng.uniform_pm1_f32(rng.hi32(rng.word(key, C.SLOT_PUSH_Y)))
        S["vx"] = np.where(pm, S["vx"] + f32(cfg.push_vel) * ux, S["vx"]).astype(f32)
        S["vy"] = np.where(pm, S["vy"] + f32(cfg.push_vel) * uy, S["vy"]).astype(f32)

    # PD torques (Sec. 3.2), 4 substeps (App. A.1.1).  The stand-in consumes the fp32
    # evaluation; the reward uses the float64 torque of the last substep.
    qdef32 = cfg.q_def.astype(f32)[:, None]
    qstar32 = qdef32 + f32(cfg.action_scale) * a32
    qstar64 = cfg.q_def.astype(np.float64)[:, None] + cfg.action_scale * a64
    tau64 = None
    for k in range(cfg.decimation):
        tau32 = f32(cfg.kp) * (qstar32 - S["q"]) - f32(cfg.kd) * S["qd"]
        if k == cfg.decimation - 1:
            tau64 = pd_torque(qstar64, S["q"], S["qd"], cfg.kp, cfg.kd)
        standin.substep(S, tau32, k, key, cfg.sim_dt)

    eplen_new = S["eplen"] + 1
    contact_prev = S["contact"]
    contact = contact_schedule(env, eplen_new)
    first = (contact & ~contact_prev) & 0xF
    S["tair"] = S["tair"] + f32(cfg.dt)                 # fp32 bookkeeping, exact on both sides
    tair64 = S["tair"].astype(np.float64)
    first_f = np.stack([(first >> f) & 1 for f in range(4)]).astype(np.float64)
    cont_f = np.stack([(contact >> f) & 1 for f in range(4)]).astype(bool)
    S["tair"] = np.where(cont_f, f32(0.0), S["tair"]).astype(f32)

    crash = rng.hi32(rng.word(key, C.SLOT_CRASH)) < np.uint64(cfg.crash_threshold)
    n_coll = rng.mulhi32(rng.hi32(rng.word(key, C.SLOT_COLLISIONS)), 3).astype(np.float64)

    # Reward: Table 2 (App. A.3), weights times dt.
    d = lambda a: np.asarray(a, np.float64)
    r_terms = reward_terms(
        v=(d(S["vx"]), d(S["vy"]), d(S["vz"])), w=(d(S["wx"]), d(S["wy"]), d(S["wz"])),
        cmd=(d(S["cmdx"]), d(S["cmdy"]), d(S["cmdw"])), qd=d(S["qd"]), qd_prev=qd_old64,
        tau=tau64, a=a64, a_prev=ap64, n_coll=n_coll, tair=tair64, first=first_f, dt=cfg.dt)
    reward = cfg.dt * r_terms.sum(0)

    # Termination (Sec. 3.2) and time-out (Sec. 2.2.1); bootstrap (Sec. 2.2.2).
    done, timeout = termination(eplen_new, crash, cfg.max_episode_len)
    reward = bootstrap_timeout(reward, values, timeout, cfg.gamma)

    # Curriculum (Sec. 3.1), decided in float64 from the fp32 pre-reset position.
    promote, demote, d2, thr = curriculum_predicates(cfg, S["px"], S["py"], S["cmdx"], S["cmdy"])
    loop = rng.mulhi32(rng.hi32(rng.word(key, C.SLOT_LOOPBACK)), cfg.num_levels)
    level_new = curriculum_level(S["level"], promote, demote, loop, cfg.num_levels)
    pre_reset = {"px": S["px"].copy(), "py": S["py"].copy(), "promote": promote & done,
                 "demote": demote & ~promote & done, "d2": d2, "thr": thr}

    S["ap"] = a32.copy()
    S["eplen"] = eplen_new
    S["contact"] = contact
    reset_state(cfg, S, done, key, level_new)

    obs = observe(cfg, hf, S, env, key)
    level = S["level"].astype(np.int32)
    terrain_idx = (S["level"] * cfg.num_cols + env % cfg.num_cols).astype(np.int32)
    sf2, si2 = pack(S)
    return {"sf": sf2, "si": si2, "obs": obs, "reward": reward, "done": done.astype(np.uint8),
            "timeout": timeout.astype(np.uint8), "level": level, "terrain_idx": terrain_idx,
            "tau": tau64.T, "pre_reset": pre_reset, "reward_terms": r_terms}
