"""Pins of the oracle's random numbers and GAE (CPU only).

RNG: the published SplitMix64 outputs and the moments of the derived variates.
GAE: closed forms (lambda = 0, lambda = 1, gamma = 0), the episode-end cut, and the direct
sum sum_l (gamma lambda)^l delta_{t+l} (a second formula, not the recursion).
"""
import os

import numpy as np
import pytest

from oracle import gae as G
from oracle import rng

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_ints(name):
    out = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            out.append(int(line, 16))
    return out


def test_splitmix64_published_outputs():
    want = _golden_ints("splitmix64_seed0.txt")
    assert [rng.word(0, k) for k in range(3)] == want
    arr = rng.word(np.zeros(3, np.uint64), np.arange(3))
    assert [int(x) for x in arr] == want


def test_mix64_array_matches_int():
    xs = [0, 1, 2 ** 63, 2 ** 64 - 1, 0x123456789ABCDEF0]
    arr = rng.mix64(np.array(xs, dtype=np.uint64))
    assert [int(a) for a in arr] == [rng.mix64(x) for x in xs]


def test_keys_distinct():
    env = np.arange(4096)
    ks = set()
    for it in range(3):
        for t in range(8):
            ks.update(int(k) for k in rng.key(7, rng.STREAM_ENV, it, t, env))
    assert len(ks) == 3 * 8 * 4096
    assert int(rng.key(7, rng.STREAM_ENV, 0, 0, 5)) != int(rng.key(7, rng.STREAM_ACT, 0, 0, 5))


def test_uniform_and_mulhi_moments():
    w = rng.word(rng.key(1, 1, 0, 0, np.arange(200000)), 3)
    u = rng.uniform01_f32(rng.hi32(w))
    assert u.dtype == np.float32 and u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    pm = rng.uniform_pm1_f32(rng.hi32(w))
    assert pm.min() >= -1 and pm.max() < 1
    # exactness: 2u - 1 in fp32 equals the float64 value
    assert np.array_equal(pm.astype(np.float64), 2 * u.astype(np.float64) - 1)
    c = np.bincount(rng.mulhi32(rng.hi32(w), 10), minlength=10)
    assert c.min() > 19000 and c.max() < 21000


def test_irwin_hall_and_box_muller_moments():
    w = rng.word(rng.key(2, 1, 0, 0, np.arange(400000)), 0)
    x = rng.irwin_hall_f32(w).astype(np.float64)
    assert abs(x.mean()) < 0.01 and abs(x.var() - 1) < 0.01
    assert abs(x).max() <= np.sqrt(3) * 2 + 1e-3          # Irwin-Hall(4) support
    # exact variance of the scaled sum: IH_SCALE^2 (2^32 - 1) / 3 ~= 1
    assert abs(float(rng.IH_SCALE) ** 2 * (2 ** 32 - 1) / 3 - 1) < 1e-6
    z = rng.box_muller_f64(w)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert abs((np.abs(z) < 1.959964).mean() - 0.95) < 0.003


def _direct_gae(rew, val, last, done, gamma, lam):
    """A_t = sum_l (gamma lambda)^l prod_{j<l} (1 - d_{t+j}) delta_{t+l}."""
    T, N = rew.shape
    vnext = np.vstack([val[1:], last[None]])
    delta = rew + gamma * (1 - done) * vnext - val
    A = np.zeros((T, N))
    for t in range(T):
        alive = np.ones(N)
        for l in range(T - t):
            A[t] += (gamma * lam) ** l * alive * delta[t + l]
            alive = alive * (1 - done[t + l])
    return A


@pytest.fixture
def traj():
    rs = np.random.default_rng(0)
    T, N = 7, 33
    return (rs.normal(size=(T, N)), rs.normal(size=(T, N)), rs.normal(size=N),
            (rs.random((T, N)) < 0.2).astype(np.float64))


def test_gae_lambda0_is_td_residual(traj):
    r, v, last, d = traj
    A, R = G.gae(r, v, last, d, 0.99, 0.0)
    vnext = np.vstack([v[1:], last[None]])
    np.testing.assert_allclose(A, r + 0.99 * (1 - d) * vnext - v, rtol=0, atol=1e-12)
    np.testing.assert_allclose(R, A + v, atol=1e-12)


def test_gae_lambda1_is_discounted_return_minus_value(traj):
    r, v, last, _ = traj
    T = r.shape[0]
    A, _ = G.gae(r, v, last, np.zeros_like(r), 0.97, 1.0)
    for t in range(T):
        ret = sum(0.97 ** k * r[t + k] for k in range(T - t)) + 0.97 ** (T - t) * last
        np.testing.assert_allclose(A[t], ret - v[t], atol=1e-12)


def test_gae_gamma0(traj):
    r, v, last, d = traj
    A, _ = G.gae(r, v, last, d, 0.0, 0.95)
    np.testing.assert_allclose(A, r - v, atol=1e-12)


def test_gae_done_cuts_recursion(traj):
    r, v, last, _ = traj
    d = np.zeros_like(r)
    d[3] = 1
    A, _ = G.gae(r, v, last, d, 0.99, 1.0)
    np.testing.assert_allclose(A[3], r[3] - v[3], atol=1e-12)


@pytest.mark.parametrize("gamma,lam", [(0.99, 0.95), (0.9, 0.5), (1.0, 1.0)])
def test_gae_matches_direct_sum(traj, gamma, lam):
    r, v, last, d = traj
    A, _ = G.gae(r, v, last, d, gamma, lam)
    np.testing.assert_allclose(A, _direct_gae(r, v, last, d, gamma, lam), atol=1e-12)


def test_gae_brute_force_t2_by_hand():
    # T = 2, one env, no done: A_1 = r1 + g V2 - V1; A_0 = (r0 + g V1 - V0) + g l A_1
    r = np.array([[1.0], [2.0]])
    v = np.array([[0.5], [0.25]])
    A, R = G.gae(r, v, np.array([4.0]), np.zeros((2, 1)), 0.5, 0.5)
    a1 = 2.0 + 0.5 * 4.0 - 0.25
    a0 = (1.0 + 0.5 * 0.25 - 0.5) + 0.25 * a1
    assert A[1, 0] == a1 and A[0, 0] == a0 and R[0, 0] == a0 + 0.5


def test_normalize():
    x = np.random.default_rng(3).normal(2.0, 5.0, 1000)
    y, m, s = G.normalize(x)
    assert abs(y.mean()) < 1e-12 and abs(y.std() - 1) < 1e-6
    assert abs(m - x.mean()) < 1e-12 and abs(s - x.std(ddof=0)) < 1e-12
