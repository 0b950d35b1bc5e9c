"""The CUDA terrain family (rl_terrain_generate) against the oracle's (oracle/terrain.py): every
grid point, on the rough-terrain workload's 10 x 20 tile grid and on a small grid of 4 m tiles,
within fp32 rounding of the float64 oracle (the random kinds draw the same counter-based words).  A config whose stair width is not a whole number of
cells is refused, and a learner trains on the generated field."""
import numpy as np
import pytest
import torch

from oracle import terrain as OT
from paper_2109_11978_b300 import api, synth
from tests.helpers import lib_config, obs_dims, workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("levels,cols,tile,seed", [(10, 20, 8.0, 0), (3, 9, 4.0, 11)])
def test_terrain_matches_oracle(levels, cols, tile, seed):
    cfg = api.default_config(num_levels=levels, num_cols=cols, tile_size=tile, seed=seed)
    got = api.rl_terrain_generate(cfg).cpu().numpy().astype(np.float64)
    want = OT.generate(levels, cols, cfg.tile_size, cfg.hf_res, cfg.seed)
    assert got.shape == want.shape
    err = np.abs(got - want)
    assert np.all(err <= 1e-6 + 2e-6 * np.abs(want)), err.max()
    # the random kinds draw the same counter-based words: equal to fp32 rounding as well
    c = int(round(cfg.tile_size / cfg.hf_res))
    for k in range(cols):
        if OT.KINDS[k % 7] in ("rough", "obstacles"):
            assert np.max(np.abs(got[:, k * c:(k + 1) * c] - want[:, k * c:(k + 1) * c])) <= 1e-7


def test_refuses_fractional_cells():
    cfg = api.default_config(hf_res=0.07)
    with pytest.raises(api.RLError):
        api.rl_terrain_generate(cfg)


def test_learner_trains_on_generated_terrain():
    w = workload("small_rough", precision=1)
    cfg = lib_config(w)
    hf = api.rl_terrain_generate(cfg).cpu().numpy()
    O, _ = obs_dims(w)
    params = synth.xavier_params(w["seed"] + 1, O, w["hidden"], 12, log_std=-0.3, bias_scale=0.1)
    L = api.Learner(cfg, hf, params)
    for _ in range(2):
        L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    assert api.rl_last_device_status(L.ctx) == 0
    obs = L.storage(0).float()
    assert torch.isfinite(obs).all()
    L.close()
