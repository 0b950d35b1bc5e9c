"""Procedural terrain family of Sec. 3.1 (terrain types of Fig. 2, difficulty by curriculum level).

TEST INFRASTRUCTURE ONLY: a plain float64 numpy restatement that the CUDA terrain generator is
checked against; it shares no code with it and nothing on the product path imports it.

What the paper fixes (Sec. 3.1, Fig. 2): five terrain types (flat, sloped, randomly rough,
discrete obstacles, stairs) on square tiles of 8 m; slopes and stairs built as pyramids so that
they can be crossed in every direction; rough terrain with 0.1 m of height variation; stairs
0.3 m wide; discrete obstacles up to +-0.2 m; with the level, the step height of stairs and
obstacles grows from 0.05 m to 0.20 m and the inclination of slopes from 0 to 25 deg.

Readings (the paper is silent on them):
* the heightfield is the curriculum grid of the env: tile rows are levels (x), tile columns are
  terrain kinds (y); column k has kind KINDS[k % 7] (pyramids going up and pits going down for
  slopes and stairs, since robots both climb and descend them);
* the difficulty of level l is d = l / (L - 1) (0 for a single level), linear in between;
* pyramids: e = the grid distance in cells from the tile border, min(a, b, c - a, c - b) for the
  in-tile grid index (a, b) of a tile of c cells, capped at c/2 - P with P = 1 m in cells (a flat
  2 m x 2 m top or bottom where the robot spawns); slope height +-tan(25 deg d) e res; stairs
  height +-s (e // W) with s = 0.05 + 0.15 d and W = 0.3 m in cells;
* rough: 0.1 (u - 0.5) per grid point, u uniform on [0, 1) from the counter generator;
* obstacles: blocks of 1 m (B cells) of height hmax * uniform(-1, 1), hmax = 0.05 + 0.15 d; the
  blocks under the central 2 m platform are flat;
* random words: key (seed, terrain stream, level, column, 0) slot a c + b for rough, key
  (seed, terrain stream, level, column, 1) slot (a // B) (c // B) + b // B for obstacles.
"""
import numpy as np

from . import rng as R

KINDS = ("flat", "slope_up", "slope_down", "rough", "obstacles", "stairs_up", "stairs_down")
MAX_SLOPE_DEG = 25.0         # Sec. 3.1: inclination 0 -> 25 deg
STEP_MIN, STEP_MAX = 0.05, 0.20   # Sec. 3.1: step height 5 cm -> 20 cm (stairs, obstacles)
STAIR_WIDTH = 0.3            # Fig. 2 (c)
ROUGH_RANGE = 0.1            # Fig. 2 (a): variations of 0.1 m
PLATFORM_HALF = 1.0          # reading: flat 2 m x 2 m spawn platform
BLOCK = 1.0                  # reading: obstacle block size


def cells(length, res):
    """length / res as an exact integer number of cells (raises if it is not one)."""
    n = int(round(length / res))
    if abs(n * res - length) > 1e-6 * max(1.0, length):
        raise ValueError(f"{length} m is not a whole number of {res} m cells")
    return n


def generate(num_levels, num_cols, tile_size, hf_res, seed):
    """Heightfield [num_levels c][num_cols c] (float64, metres), c = tile_size / hf_res."""
    c = cells(tile_size, hf_res)
    P, W, B = cells(PLATFORM_HALF, hf_res), cells(STAIR_WIDTH, hf_res), cells(BLOCK, hf_res)
    if c % 2 or c % B or c // 2 < P:
        raise ValueError("tile must be an even number of cells, whole blocks and hold the platform")
    a = np.arange(c)[:, None]
    b = np.arange(c)[None, :]
    e = np.minimum(np.minimum(a, b), np.minimum(c - a, c - b))          # cells to the tile border
    e = np.minimum(e, c // 2 - P)
    nb = c // B
    blk_a, blk_b = a // B, b // B
    centre = (np.abs(2 * blk_a + 1 - nb) <= 1) & (np.abs(2 * blk_b + 1 - nb) <= 1)
    hf = np.zeros((num_levels * c, num_cols * c), dtype=np.float64)
    for lvl in range(num_levels):
        d = lvl / (num_levels - 1) if num_levels > 1 else 0.0
        step = STEP_MIN + (STEP_MAX - STEP_MIN) * d
        for k in range(num_cols):
            kind = KINDS[k % len(KINDS)]
            if kind == "flat":
                h = np.zeros((c, c))
            elif kind in ("slope_up", "slope_down"):
                h = np.tan(np.deg2rad(MAX_SLOPE_DEG * d)) * e * hf_res
                h = h if kind == "slope_up" else -h
            elif kind in ("stairs_up", "stairs_down"):
                h = step * (e // W)
                h = h if kind == "stairs_up" else -h
            elif kind == "rough":
                key = R.key(seed, R.STREAM_TERRAIN, lvl, k, 0)
                w = R.word(key, (a * c + b).astype(np.uint64).ravel())
                u = R.uniform01_f32(R.hi32(w)).astype(np.float64).reshape(c, c)
                h = ROUGH_RANGE * (u - 0.5)
            else:   # obstacles
                key = R.key(seed, R.STREAM_TERRAIN, lvl, k, 1)
                slot = (blk_a * nb + blk_b) * np.ones_like(b)
                w = R.word(key, slot.astype(np.uint64).ravel())
                u = R.uniform_pm1_f32(R.hi32(w)).astype(np.float64).reshape(c, c)
                h = np.where(centre, 0.0, step * u)
            hf[lvl * c:(lvl + 1) * c, k * c:(k + 1) * c] = h
    return hf
