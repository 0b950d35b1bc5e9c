"""Pins of the oracle's terrain family (Sec. 3.1, Fig. 2) against the numbers the paper prints:
25 deg slopes, steps from 0.05 m to 0.20 m, 0.3 m wide stairs, 0.1 m rough variation, obstacles of
up to +-0.2 m, pyramids traversable from every side, difficulty growing with the level."""
import numpy as np
import pytest

from oracle import terrain as T

L, C, TILE, RES = 10, 14, 8.0, 0.1
c = 80


@pytest.fixture(scope="module")
def hf():
    return T.generate(L, C, TILE, RES, seed=3)


def tile(hf, lvl, k):
    return hf[lvl * c:(lvl + 1) * c, k * c:(k + 1) * c]


def kind_cols(name):
    return [k for k in range(C) if T.KINDS[k % 7] == name]


def test_layout_and_flat(hf):
    assert hf.shape == (L * c, C * c)
    for k in kind_cols("flat"):
        assert not np.any(tile(hf, 0, k)) and not np.any(tile(hf, L - 1, k))


def test_slopes_rise_at_the_level_inclination(hf):
    k_up, k_dn = kind_cols("slope_up")[0], kind_cols("slope_down")[0]
    assert not np.any(tile(hf, 0, k_up))                           # level 0: 0 deg
    for lvl in (3, L - 1):
        t = tile(hf, lvl, k_up)
        theta = np.deg2rad(25.0 * lvl / (L - 1))
        row = t[c // 2, :c // 2 - 10 + 1]                          # border -> platform edge, 3 m
        assert np.allclose(np.diff(row), np.tan(theta) * RES, rtol=1e-12, atol=0)
        assert t.max() == pytest.approx(np.tan(theta) * 3.0, rel=1e-12)
        assert np.all(t[c // 2 - 10:c // 2 + 10, c // 2 - 10:c // 2 + 10] == t.max())   # 2 m platform
        assert np.array_equal(tile(hf, lvl, k_dn), -t)             # the pit mirrors the pyramid
        assert np.all(t[0, :] == 0) and np.all(t[:, 0] == 0)       # meets the next tile at 0
    assert tile(hf, L - 1, k_up).max() == pytest.approx(np.tan(np.deg2rad(25.0)) * 3.0, rel=1e-12)


def test_stairs_step_height_and_width(hf):
    k = kind_cols("stairs_up")[0]
    for lvl, step in ((0, 0.05), (L - 1, 0.20)):
        t = tile(hf, lvl, k)
        n = t / step
        assert np.allclose(n, np.round(n), atol=1e-9)               # whole steps
        assert np.array_equal(np.unique(np.round(n)), np.arange(11))  # 10 steps up to the platform
        row = np.round(t[c // 2, :c // 2] / step)
        assert np.array_equal(row[:30], np.repeat(np.arange(10), 3))  # 0.3 m treads
    assert np.array_equal(tile(hf, 4, kind_cols("stairs_down")[0]), -tile(hf, 4, k))


def test_rough_variation(hf):
    for k in kind_cols("rough"):
        for lvl in (0, L - 1):
            t = tile(hf, lvl, k)
            assert t.min() >= -0.05 and t.max() < 0.05
            assert abs(t.std() - 0.1 / np.sqrt(12)) < 0.003           # uniform over 0.1 m
            assert np.mean(t[:, 1:] != t[:, :-1]) > 0.99              # drawn per grid point


def test_obstacle_blocks(hf):
    k = kind_cols("obstacles")[0]
    for lvl in (0, 5, L - 1):
        step = 0.05 + 0.15 * lvl / (L - 1)
        t = tile(hf, lvl, k)
        blocks = t.reshape(8, 10, 8, 10)
        assert np.all(blocks == blocks[:, :1, :, :1])                # constant on 1 m blocks
        assert np.all(np.abs(t) <= step)
        assert not np.any(t[30:50, 30:50])                          # the central 2 m blocks
        vals = blocks[:, 0, :, 0]
        assert len(np.unique(vals)) >= 55 and np.abs(vals).max() > 0.8 * step
    assert np.abs(tile(hf, L - 1, k)).max() <= 0.2


def test_seed_and_whole_cells():
    a = T.generate(2, 7, TILE, RES, seed=1)
    assert np.array_equal(a, T.generate(2, 7, TILE, RES, seed=1))
    b = T.generate(2, 7, TILE, RES, seed=2)
    assert not np.array_equal(a, b)
    assert np.array_equal(a[:, :3 * c], b[:, :3 * c])                # only random kinds change
    with pytest.raises(ValueError):
        T.generate(2, 7, TILE, 0.07, seed=1)
