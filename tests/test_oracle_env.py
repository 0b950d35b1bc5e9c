"""Pins of the oracle's env-side math (CPU only).

* Table 2 reward weights and Table 4 noise scales against the fixtures transcribed from the
  paper (tests/golden/);
* reward terms on hand-computed examples (perfect tracking gives dt (1 + 0.5) = 0.03; every
  term isolated by zeroing the others);
* PD torque by hand (Sec. 3.2);
* height samples: exact on the flat first row of tiles, exact for an affine heightfield,
  equal to the stored value at grid nodes, axes swapped by a quarter turn of the heading;
* curriculum: exhaustive truth table of the level update, the strict 4 m border and the
  half-commanded-distance threshold (Sec. 3.1);
* termination / time-out / bootstrap (Sec. 2.2.1, 2.2.2);
* invariants of a full step on diverse states, noise bounds (Table 4), pushes (Sec. 3.3).
"""
import os

import numpy as np
import pytest

from oracle import config as C
from oracle import env as E
from oracle import rng
from paper_2109_11978_b300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kv(name):
    d = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            d[k] = float(v)
    return d


def test_table2_weights():
    t = _kv("table2_reward_weights.txt")
    assert (C.W_LIN_VEL, C.W_ANG_VEL, C.W_VZ, C.W_WXY, C.W_JOINT, C.W_TORQUE, C.W_ACTION_RATE,
            C.W_COLLISION, C.W_AIR_TIME) == (
        t["lin_vel_tracking"], t["ang_vel_tracking"], t["lin_vel_z_penalty"], t["ang_vel_xy_penalty"],
        t["joint_motion"], t["joint_torques"], t["action_rate"], t["collisions"], t["feet_air_time"])
    assert C.PHI_SCALE == t["phi_denominator"] and C.AIR_TIME_TARGET == t["air_time_target"]


def test_table4_noise_layout():
    t = _kv("table4_noise.txt")
    s = C.EnvConfig().noise_scales()
    assert s.shape == (235,)
    np.testing.assert_array_equal(s[0:3], t["base_linear_velocity"])
    np.testing.assert_array_equal(s[3:6], t["base_angular_velocity"])
    np.testing.assert_array_equal(s[6:9], t["projected_gravity"])
    np.testing.assert_array_equal(s[9:11], t["commanded_base_linear_velocity"])
    np.testing.assert_array_equal(s[11], t["commanded_base_angular_velocity"])
    np.testing.assert_array_equal(s[12:24], t["joint_positions"])
    np.testing.assert_array_equal(s[24:36], t["joint_velocities"])
    np.testing.assert_array_equal(s[48:], t["measured_terrain_heights"])


def _zero_reward_inputs(n=1):
    z = np.zeros(n)
    return dict(v=(z, z, z), w=(z, z, z), cmd=(z, z, z), qd=np.zeros((12, n)), qd_prev=np.zeros((12, n)),
                tau=np.zeros((12, n)), a=np.zeros((12, n)), a_prev=np.zeros((12, n)), n_coll=z,
                tair=np.zeros((4, n)), first=np.zeros((4, n)), dt=0.02)


def test_reward_perfect_tracking_is_0_03():
    kw = _zero_reward_inputs()
    kw["cmd"] = (np.array([0.7]), np.array([-0.3]), np.array([0.4]))
    kw["v"] = (np.array([0.7]), np.array([-0.3]), np.array([0.0]))
    kw["w"] = (np.array([0.0]), np.array([0.0]), np.array([0.4]))
    r = 0.02 * E.reward_terms(**kw).sum(0)
    assert abs(r[0] - 0.03) < 1e-15


@pytest.mark.parametrize("case,term,value", [
    ("lin_err_0.5", 0, np.exp(-1.0)),       # |v* - v|^2 = 0.25 -> phi = e^-1
    ("ang_err_0.5", 1, 0.5 * np.exp(-1.0)),
    ("vz_0.5", 2, -4.0 * 0.25),
    ("wxy_0.3_0.4", 3, -0.05 * 0.25),
    ("qdd_1", 4, -0.001 * (1.0 + 0.02 ** 2)),
    ("tau_10", 5, -0.00002 * 100.0),
    ("rate_2", 6, -0.25 * 4.0),
    ("coll_2", 7, -0.001 * 2.0),
    ("air_0.7_two_feet", 8, 2.0 * (0.2 + 0.2)),
])
def test_reward_terms_isolated(case, term, value):
    kw = _zero_reward_inputs()
    one = np.array([1.0])
    if case == "lin_err_0.5":
        kw["cmd"] = (0.5 * one, 0 * one, 0 * one)
    elif case == "ang_err_0.5":
        kw["cmd"] = (0 * one, 0 * one, 0.5 * one)
    elif case == "vz_0.5":
        kw["v"] = (0 * one, 0 * one, 0.5 * one)
    elif case == "wxy_0.3_0.4":
        kw["w"] = (0.3 * one, 0.4 * one, 0 * one)
    elif case == "qdd_1":
        kw["qd"][3] = 0.02                    # qd_prev = 0 -> qdd = 0.02 / 0.02 = 1
    elif case == "tau_10":
        kw["tau"][5] = 10.0
    elif case == "rate_2":
        kw["a"][0], kw["a_prev"][0] = 1.5, -0.5
    elif case == "coll_2":
        kw["n_coll"] = 2 * one
    elif case == "air_0.7_two_feet":
        kw["tair"][:] = 0.7
        kw["first"][1] = kw["first"][2] = 1
    terms = E.reward_terms(**kw)
    base = np.array([np.exp(-0.0), 0.5, 0, 0, 0, 0, 0, 0, 0])
    if term in (0, 1):
        base[term] = value
    else:
        base[term] = value
    if case == "lin_err_0.5":
        base[1] = 0.5
    np.testing.assert_allclose(terms[:, 0], base, rtol=1e-14, atol=1e-16)


def test_pd_torque_by_hand():
    tau = E.pd_torque(np.array([0.5]), np.array([0.2]), np.array([1.0]), 80.0, 2.0)
    assert abs(tau[0] - (80.0 * 0.3 - 2.0)) < 1e-12


def _obs_cfg(**kw):
    cfg = C.EnvConfig(num_envs=kw.pop("n", 8), noise_on=False, push_on=False, **kw)
    return cfg


def _state_for_heights(cfg, level, px, py, c, s, z=0.6):
    n = len(px)
    S = E.unpack(*synth.random_env_state(0, n))
    S["level"] = np.asarray(level, np.int64)
    S["px"], S["py"] = np.asarray(px, np.float32), np.asarray(py, np.float32)
    S["hc"], S["hs"] = np.asarray(c, np.float32), np.asarray(s, np.float32)
    S["z"] = np.full(n, z, np.float32)
    return S


def test_heights_flat_first_row_equal_base_height():
    cfg = _obs_cfg()
    hf = synth.heightfield(3)
    n = cfg.num_envs
    rs = np.random.default_rng(0)
    S = _state_for_heights(cfg, np.zeros(n), rs.uniform(-3, 3, n), rs.uniform(-3, 3, n),
                           np.ones(n), np.zeros(n), z=0.55)
    o = E.observe(cfg, hf, S, np.arange(n), None)
    assert np.all(o[:, 48:] == np.float64(np.float32(0.55)))


def test_heights_affine_terrain_exact():
    cfg = _obs_cfg()
    a, b, c0 = 0.01, -0.004, 0.3           # per cell
    hf = synth.affine_heightfield(cfg.hf_shape, a, b, c0).astype(np.float64)
    rs = np.random.default_rng(1)
    n = cfg.num_envs
    yaw = rs.uniform(-np.pi, np.pi, n)
    S = _state_for_heights(cfg, rs.integers(1, 9, n), rs.uniform(-3, 3, n), rs.uniform(-3, 3, n),
                           np.cos(yaw), np.sin(yaw))
    env = np.arange(n)
    o = E.observe(cfg, hf.astype(np.float32), S, env, None)
    ox, oy = E.spawn_origin(cfg, S["level"].astype(np.float64), env)
    gx, gy = E.grid_offsets(cfg)
    c, s = S["hc"].astype(np.float64), S["hs"].astype(np.float64)
    X = ox[:, None] + S["px"].astype(np.float64)[:, None] + c[:, None] * gx - s[:, None] * gy
    Y = oy[:, None] + S["py"].astype(np.float64)[:, None] + s[:, None] * gx + c[:, None] * gy
    # fp32 storage of the affine field limits agreement to fp32 rounding of its values
    want = S["z"].astype(np.float64)[:, None] - (a * X / cfg.hf_res + b * Y / cfg.hf_res + c0)
    np.testing.assert_allclose(o[:, 48:], want, atol=2e-7)


def test_heights_at_nodes_and_quarter_turn():
    cfg = _obs_cfg(n=2)
    hf = synth.heightfield(7)
    env = np.arange(2)
    # heading along +x: sample (ix, iy) sits on node (i0 + ix - 8, j0 + iy - 5)
    S = _state_for_heights(cfg, [4, 4], [0.0, 0.0], [0.0, 0.0], [1.0, 0.0], [0.0, 1.0])
    o = E.observe(cfg, hf, S, env, None)
    i0, j0 = 4 * 80 + 40, (0 + 0.5) * 80
    j0 = int(j0)
    h = o[0, 48:].reshape(cfg.grid_y, cfg.grid_x)             # [iy, ix]
    for iy in range(cfg.grid_y):
        for ix in range(cfg.grid_x):
            node = hf[i0 + ix - 8, j0 + iy - 5]
            assert abs(h[iy, ix] - (np.float64(np.float32(0.6)) - node)) < 1e-12
    # env 1 is in column 1 and turned by +90 degrees: body x points to world +y
    j1 = int(1.5 * 80)
    h1 = o[1, 48:].reshape(cfg.grid_y, cfg.grid_x)
    for iy in range(cfg.grid_y):
        for ix in range(cfg.grid_x):
            node = hf[i0 - (iy - 5), j1 + (ix - 8)]
            assert abs(h1[iy, ix] - (np.float64(np.float32(0.6)) - node)) < 1e-6


def test_curriculum_truth_table():
    L, loop = 10, 3
    # (level, promote, demote) -> new level, worked by hand from Sec. 3.1
    table = {(0, 0, 0): 0, (0, 0, 1): 0, (0, 1, 0): 1, (0, 1, 1): 1,
             (5, 0, 0): 5, (5, 0, 1): 4, (5, 1, 0): 6, (5, 1, 1): 6,
             (9, 0, 0): 9, (9, 0, 1): 8, (9, 1, 0): loop, (9, 1, 1): loop}
    for (lv, p, d), want in table.items():
        got = E.curriculum_level(np.array([lv]), np.array([bool(p)]), np.array([bool(d)]), np.array([loop]), L)
        assert got[0] == want, (lv, p, d, got, want)


def test_curriculum_predicates_thresholds():
    cfg = C.EnvConfig()
    p, _, _, _ = E.curriculum_predicates(cfg, np.float32([4.0, 4.0001, 0.0, 2.5]),
                                         np.float32([0.0, 0.0, -4.0001, 3.2]), np.zeros(4), np.zeros(4))
    assert list(p) == [False, True, True, True]           # strict: exactly 4 m is not past the border
    # |v*| = 1 m/s over 20 s -> half distance ~ 10 m (T = 1000 * fp32(0.02))
    _, d, _, thr = E.curriculum_predicates(cfg, np.float32([9.9, 10.1, 0.0]), np.float32([0, 0, 0]),
                                           np.float32([1.0, 1.0, 0.0]), np.float32([0.0, 0.0, 0.0]))
    assert list(d) == [True, False, False]                 # zero command never demotes
    assert abs(np.sqrt(thr[0]) - 10.0) < 1e-6


def test_termination_and_bootstrap():
    done, timeout = E.termination(np.array([999, 1000, 1000, 5]), np.array([False, False, True, True]), 1000)
    assert list(done) == [False, True, True, True]
    assert list(timeout) == [False, True, False, False]
    r = E.bootstrap_timeout(np.zeros(4), np.full(4, 2.0), timeout, 0.99)
    assert list(r) == [0.0, 0.99 * 2.0, 0.0, 0.0]


def _run_step(cfg, seed=0, n=256):
    hf = synth.heightfield(1)
    sf, si = synth.random_env_state(seed, n)
    a = np.random.default_rng(seed).normal(size=(n, 12)).astype(np.float32)
    v = np.random.default_rng(seed + 1).normal(size=n)
    return sf, si, a, v, E.step(cfg, hf, sf, si, a, v, 3, 5)


def test_step_invariants():
    cfg = C.EnvConfig(num_envs=256, crash_threshold=2 ** 28)      # ~6 % crashes to exercise resets
    sf, si, a, v, r = _run_step(cfg)
    n = sf.shape[1]
    env = np.arange(n)
    assert r["sf"].dtype == np.float32 and r["obs"].shape == (n, 235)
    lv = r["level"]
    assert lv.min() >= 0 and lv.max() < cfg.num_levels
    assert np.array_equal(r["terrain_idx"], lv * cfg.num_cols + env % cfg.num_cols)
    done = r["done"].astype(bool)
    assert done.any() and (~done).any()
    S = E.unpack(r["sf"], r["si"])
    assert np.all(S["px"][done] == 0) and np.all(S["eplen"][done] == 0) and np.all(S["ap"][:, done] == 0)
    assert np.array_equal(S["eplen"][~done], si[E.I_EPLEN][~done] + 1)
    assert np.array_equal(S["ap"][:, ~done], a.T[:, ~done])
    assert np.array_equal(r["timeout"].astype(bool), (si[E.I_EPLEN] + 1 >= 1000) & ~(done & ~r["timeout"].astype(bool)))
    np.testing.assert_allclose(S["hc"] ** 2 + S["hs"] ** 2, 1.0, atol=1e-6)
    # levels change only for reset robots
    assert np.array_equal(lv[~done], si[E.I_LEVEL][~done])
    # promotions/demotions as predicted by the pre-reset decision
    pr = r["pre_reset"]
    assert np.all(lv[pr["demote"]] == np.maximum(si[E.I_LEVEL][pr["demote"]] - 1, 0))


def test_step_is_deterministic_and_fp32():
    cfg = C.EnvConfig(num_envs=64)
    a1 = _run_step(cfg, 2, 64)[-1]
    a2 = _run_step(cfg, 2, 64)[-1]
    assert np.array_equal(a1["sf"], a2["sf"]) and np.array_equal(a1["obs"], a2["obs"])


def test_observation_noise_bounds():
    on = _run_step(C.EnvConfig(num_envs=128, noise_on=True), 4, 128)[-1]
    off = _run_step(C.EnvConfig(num_envs=128, noise_on=False), 4, 128)[-1]
    assert np.array_equal(on["sf"], off["sf"])
    diff = np.abs(on["obs"] - off["obs"])
    scales = C.EnvConfig().noise_scales()
    assert np.all(diff <= scales[None, :] + 1e-12)
    assert np.all(diff[:, 9:12] == 0) and np.all(diff[:, 36:48] == 0)
    assert np.all(diff[:, 24:36].max(0) > 0.5 * 1.5)     # noise actually drawn


def test_pushes_every_interval():
    cfg_on = C.EnvConfig(num_envs=64, push_on=True)
    cfg_off = C.EnvConfig(num_envs=64, push_on=False)
    hf = synth.heightfield(1)
    sf, si = synth.random_env_state(9, 64)
    si[E.I_EPLEN, :32] = 500
    si[E.I_EPLEN, 32:] = 499
    a = np.zeros((64, 12), np.float32)
    on = E.step(cfg_on, hf, sf, si, a, np.zeros(64), 0, 0)
    off = E.step(cfg_off, hf, sf, si, a, np.zeros(64), 0, 0)
    moved = np.any(on["sf"] != off["sf"], axis=0)
    assert moved[:32].all() and not moved[32:].any()


def test_initial_state():
    cfg = C.EnvConfig(num_envs=500)
    sf, si = E.initial_state(cfg)
    assert np.all(si[E.I_LEVEL] == 0)
    assert si[E.I_EPLEN].min() >= 0 and si[E.I_EPLEN].max() < 1000 and len(np.unique(si[E.I_EPLEN])) > 300
    np.testing.assert_allclose(sf[E.F_HC] ** 2 + sf[E.F_HS] ** 2, 1.0, atol=1e-6)
    assert np.all(np.abs(sf[E.F_CMDX:E.F_CMDW + 1]) <= 1.0)
