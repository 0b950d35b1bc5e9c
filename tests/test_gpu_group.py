"""Grouped learners: independent learners of uneven robot counts trained by one grouped CUDA
graph give exactly the results of the same learners trained one by one (the kernels are
deterministic and the learners share nothing)."""
import numpy as np
import pytest
import torch

from paper_2109_11978_b300 import api, synth
from tests.helpers import lib_config, obs_dims, workload

pytestmark = pytest.mark.gpu


def _cfgs(prec):
    out = []
    for i, n in enumerate((64, 128, 192)):
        w = workload("tiny", num_envs=n, seed=10 + i, precision=prec)
        O, _ = obs_dims(w)
        out.append((lib_config(w), synth.xavier_params(w["seed"] + 1, O, w["hidden"], 12)))
    return out


def _params(ctx, cfg):
    p = torch.empty(api.rl_param_count(cfg), device="cuda")
    api.rl_get_params(ctx, p)
    return p


@pytest.mark.parametrize("prec", [0, 1])
def test_group_graph_equals_learners_one_by_one(prec):
    cfgs = _cfgs(prec)
    g = api.rl_group_create([c for c, _ in cfgs], [None] * len(cfgs), [p for _, p in cfgs])
    solo = [api.Learner(c, None, p) for c, p in cfgs]
    for _ in range(2):
        api.rl_group_train_iteration(g, use_graph=True)
        for L in solo:
            L.train_iteration(use_graph=False)
    torch.cuda.synchronize()
    for i, ((c, _), L) in enumerate(zip(cfgs, solo)):
        ctx = api.rl_group_learner(g, i)
        assert torch.equal(_params(ctx, c), L.params()), i
        assert api.rl_get_scalars(ctx)["iteration"] == 2
        assert api.rl_last_device_status(ctx) == 0
    api.rl_group_destroy(g)
    for L in solo:
        L.close()


@pytest.mark.parametrize("cap", [16, 37])
def test_gemm_cta_cap_keeps_results(cap):
    """A learner whose GEMM launches run on at most `cap` persistent CTAs (as grouped learners'
    do) trains bit for bit like one with a CTA per SM: the cap moves tiles between CTAs, never
    changes a sum."""
    w = workload("small_rough", precision=1, epochs=2, minibatches=2)
    O, _ = obs_dims(w)
    params = synth.xavier_params(w["seed"] + 1, O, w["hidden"], 12)
    hf = synth.heightfield(w["seed"] + 2)
    A = api.Learner(lib_config(w), hf, params)
    B = api.Learner(lib_config(w), hf, params)
    api.rl_set_gemm_ctas(B.ctx, cap)
    for _ in range(2):
        A.train_iteration(use_graph=True)
        B.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    assert torch.equal(A.params(), B.params())
    assert api.rl_last_device_status(B.ctx) == 0
    with pytest.raises(api.RLError):
        api.rl_set_gemm_ctas(B.ctx, -1)
    A.close()
    B.close()
