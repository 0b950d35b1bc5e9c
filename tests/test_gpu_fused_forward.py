"""GPU parity (through the C ABI) of the fused forward of the three hidden layers
(rl_set_forward_fused): at the rollout's site and at the update's it gives the same bits as the
layer-by-layer launches, and the oracle's outputs and gradients within the BF16 tolerance; row
counts span many tiles and several waves (24576), a ragged last tile (1000, 2880) and a lone
partial tile (64).  A whole training iteration with both sites fused repeats the layered one
bit for bit, and is checked against the oracle's rollout in test_gpu_update_parity."""
import numpy as np
import pytest
import torch

from oracle import mlp as OM
from oracle import ppo as OP
from paper_2109_11978_b300 import api
from tests.gpu_helpers import _batch, _obs, _own_old_policy, _per_tensor_err, _setup
from tests.helpers import TOL_BF16, rel_err, workload

pytestmark = pytest.mark.gpu


def _act(L, xd, rows):
    out = [torch.empty((rows, 12), device="cuda"), torch.empty((rows, 12), device="cuda"),
           torch.empty(rows, device="cuda"), torch.empty(rows, device="cuda")]
    api.rl_policy_act(L.ctx, 3, xd, *out)
    v_only = torch.empty(rows, device="cuda")
    api.rl_policy_act(L.ctx, 3, xd, None, None, None, v_only)       # the critic alone: one network per launch
    torch.cuda.synchronize()
    return out + [v_only]


@pytest.mark.parametrize("rows", [4096, 1000, 64, 24576])
def test_rollout_forward_fused_equals_layers(rows):
    w = workload("rough", precision=1)
    L, params, O, Op = _setup(w)
    x, xd = _obs(rows, O, Op, 5, True)
    layered = _act(L, xd, rows)
    assert api.rl_get_forward_fused(L.ctx, 3) == 0
    api.rl_set_forward_fused(L.ctx, 3, 1)
    assert api.rl_get_forward_fused(L.ctx, 3) == 1
    fused = _act(L, xd, rows)
    for name, a, b in zip(("actions", "mu", "logp", "values", "values_alone"), layered, fused):
        assert torch.equal(a, b), name
    assert api.rl_last_device_status(L.ctx) == 0
    if rows <= 4096:
        p = OM.unflatten(params, O, w["hidden"], 12)
        ref = OM.act(p, x[:, :O], w["seed"], 0, 3)
        for k, got in zip(("actions", "mu", "logp", "values"), fused[:4]):
            assert rel_err(got.cpu().numpy(), ref[k]) < TOL_BF16, k
    L.close()


@pytest.mark.parametrize("M", [2880, 64, 24576])
def test_update_forward_fused_equals_layers(M):
    """The update's forward keeps every layer's activations for the backward: the loss gradient
    (which reads all of them) is the same bit for bit, and the oracle's within the BF16 tolerance."""
    w = workload("rough", precision=1)
    L, params, O, Op = _setup(w)
    hidden = w["hidden"]
    b, d = _batch(M, O, Op, 12, params, hidden, 43, True, kink_margin=True)
    d = _own_old_policy(L, b, d, O, params, hidden)

    def grad():
        g = torch.empty(L.n_params, device="cuda")
        api.rl_ppo_loss_grad(L.ctx, d["obs"], d["actions"], d["logp_old"], d["mu_old"], d["log_std_old"], d["v_old"],
                             d["adv"], d["ret"], g)
        torch.cuda.synchronize()
        return g

    g0 = grad()
    api.rl_set_forward_fused(L.ctx, 0, 1)
    g1 = grad()
    assert torch.equal(g0, g1)
    assert api.rl_last_device_status(L.ctx) == 0
    if M <= 2880:
        p = OM.unflatten(params, O, hidden, 12)
        _, gr, _ = OP.loss_and_grad(p, b["obs"][:, :O], b["actions"], b["logp_old"], b["mu_old"], b["log_std_old"],
                                    b["v_old"], b["adv"], b["ret"])
        errs = _per_tensor_err(g1.cpu().numpy(), OP.flat_grad(gr), (O, hidden, 12), rel_err)
        assert max(errs.values()) < TOL_BF16, errs
    L.close()


def test_training_iteration_fused_equals_layers():
    """Two learners from the same seed, one with both forward sites fused: after two training
    iterations (graph-captured) their parameters and rollout storage agree bit for bit (the episode
    statistics, summed by float atomics, to 1e-6)."""
    w = workload("small_rough", precision=1, hidden=(512, 256, 128), epochs=2, minibatches=2)
    La, _, _, _ = _setup(w)
    Lb, _, _, _ = _setup(w)
    api.rl_set_forward_fused(Lb.ctx, 0, 1)
    api.rl_set_forward_fused(Lb.ctx, 3, 1)
    for _ in range(2):
        La.train_iteration(use_graph=True)
        Lb.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    assert torch.equal(La.params(), Lb.params())
    for i, name in La.STORAGE.items():
        a, b = La.storage(i), Lb.storage(i)
        if name == "stats":
            # the env step's episode sums are float atomics, whose order varies from run to run
            assert torch.allclose(a, b, rtol=1e-6, atol=0.0)
        else:
            assert torch.equal(a, b), name
    assert api.rl_last_device_status(La.ctx) == 0 and api.rl_last_device_status(Lb.ctx) == 0
    La.close()
    Lb.close()


def test_autotune_times_the_fused_forward():
    w = workload("small_rough", precision=1, hidden=(512, 256, 128), num_envs=480)
    L, _, _, _ = _setup(w)
    rep = api.rl_autotune(L.ctx)
    sites = {s["site"]: s for s in rep["sites"]}
    for name, site in (("forward_fused", 0), ("act_forward_fused", 3)):
        assert name in sites
        assert sites[name]["cluster"] == api.rl_get_forward_fused(L.ctx, site)
    L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()


def test_set_forward_fused_rejects_invalid():
    w = workload("rough", precision=0)              # FP32: no tensor-core forward
    L, _, _, _ = _setup(w)
    with pytest.raises(api.RLError):
        api.rl_set_forward_fused(L.ctx, 0, 1)
    api.rl_set_forward_fused(L.ctx, 0, 0)
    L.close()
    w = workload("tiny", precision=1)               # two hidden layers of 64
    L, _, _, _ = _setup(w)
    for site, on in ((0, 1), (3, 1), (1, 0), (2, 1), (0, 2)):
        with pytest.raises(api.RLError):
            api.rl_set_forward_fused(L.ctx, site, on)
    with pytest.raises(api.RLError):
        api.rl_get_forward_fused(L.ctx, 1)
    L.close()


def test_fused_forward_not_used_under_a_cta_cap():
    """A learner whose GEMM CTAs are capped (grouped learners) runs its forward layer by layer: the
    fused launch takes one CTA per row tile and network."""
    w = workload("rough", precision=1)
    L, _, O, Op = _setup(w)
    api.rl_set_forward_fused(L.ctx, 3, 1)
    api.rl_set_gemm_ctas(L.ctx, 32)
    assert api.rl_get_forward_fused(L.ctx, 3) == 0
    x, xd = _obs(256, O, Op, 7, True)
    capped = _act(L, xd, 256)
    api.rl_set_gemm_ctas(L.ctx, 0)
    assert api.rl_get_forward_fused(L.ctx, 3) == 1
    fused = _act(L, xd, 256)
    for a, b in zip(capped, fused):
        assert torch.equal(a, b)
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()
