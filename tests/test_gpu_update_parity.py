"""GPU parity of the whole PPO update and of the benchmarked rollout form against the FP64 oracle.

* The epoch permutations the library draws (Sec. 2.2.1: minibatches of a shuffled batch) equal the
  oracle's bit for bit, at the tiny and at the full rough-terrain size.
* rl_ppo_update over several epochs x minibatches against oracle.ppo.update: the per-minibatch KL
  and the learning rate Algorithm 1 (App. A.4) chose, including both clamps, the divide and the
  multiply branch and the unchanged one; Adam's step count and moments after steps >= 2; the
  parameters.  FP32.
* A full training iteration of the rough-terrain form the bench times (height samples, Table 4
  noise, the policy heads fused into the env step) teacher-forced through the oracle's rollout,
  in BF16 and FP32, on the 17 x 11 and the 108-point (12 x 9) height grids.

Tolerances (relative, per tensor, |x - ref|_inf / |ref|_inf unless stated):
* FP32 Adam moments: 1e-5 (m) and 2e-5 (v, whose g^2 doubles the relative error of g);
* parameters after the update: |dp - dp_ref| <= 1e-3 sum(alpha) per element.  The oracle and the
  library agree on every gradient to ~1e-6 relative (norm-wise); from Adam's second step on, the
  step direction m_hat / sqrt(v_hat) depends on ratios of successive gradients, which turns an
  elementwise gradient error of a small element into a step error of the same relative size, so the
  bound is set a hundred times above the gradient tolerance but far below what a wrong moment, beta
  or bias correction gives (an O(1) fraction of alpha per step);
* alpha: the same branch of Algorithm 1 at every minibatch and the same value to 1e-6 (fp32
  arithmetic of alpha / 1.5, 1.5 alpha and the clamps); KL to 1e-4 relative.
"""
import numpy as np
import pytest
import torch

from oracle import config as OC
from oracle import gae as OG
from oracle import mlp as OM
from oracle import ppo as OP
from oracle.train import Learner as OLearner
from paper_2109_11978_b300 import api, synth
from tests.gpu_helpers import _batch, _segments, _setup
from tests.helpers import (TOL_BF16, TOL_FP32, lib_config, obs_dims, oracle_env_config, oracle_ppo_config, rel_err,
                           workload)

pytestmark = pytest.mark.gpu


def _oracle_perms(B, epochs, minibatches, seed, iteration):
    return np.stack([np.concatenate(OP.minibatch_indices(B, minibatches, seed, iteration, e)) for e in range(epochs)])


@pytest.mark.parametrize("name,prec", [("tiny", 0), ("rough", 1)])
def test_update_permutations_match_oracle(name, prec):
    """The shuffle of every epoch (a cycle-walking Feistel permutation keyed by seed, iteration and
    epoch) equals the oracle's bit for bit; the device status stays clean (no walk ran out)."""
    w = workload(name, precision=prec, epochs=2 if name == "tiny" else 5, minibatches=2 if name == "tiny" else 4)
    L, _, _, _ = _setup(w)
    B = w["num_envs"] * w["num_steps"]
    for it in range(2):
        L.train_iteration(use_graph=True)
        torch.cuda.synchronize()
        got = L.storage(13).cpu().numpy()
        want = _oracle_perms(B, w["epochs"], w["minibatches"], w["seed"], it)
        assert np.array_equal(got, want), it
        assert np.array_equal(np.sort(got, axis=1), np.tile(np.arange(B), (w["epochs"], 1)))
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()


def _kl_schedule(mu, log_std, groups, kls, rs):
    """mu_old = mu + d: per sample a mean offset whose closed-form KL(pi_old || pi) (equal sigmas:
    sum_j d_j^2 / (2 sigma_j^2)) is kls[g] for the samples of group g."""
    s2 = np.exp(2.0 * log_std)
    out = np.array(mu, np.float64)
    for idx, kl in zip(groups, kls):
        mag = np.sqrt(2.0 * s2 * kl / s2.size)
        out[idx] += rs.choice([-1.0, 1.0], size=(idx.size, s2.size)) * mag
    return out.astype(np.float32)


def _branches(alphas, start):
    prev, out = start, []
    for a in alphas:
        out.append("up" if a > prev * (1 + 1e-6) else "down" if a < prev * (1 - 1e-6) else "same")
        prev = a
    return out


def _check_update(L, oracle, flat0, flat_ref, alpha_ref_trace, kl_ref_trace, alpha0, dims, n_mb):
    trace = L.storage(14).cpu().numpy()[:n_mb].astype(np.float64)
    kl_gpu, a_gpu = trace[:, 0], trace[:, 1]
    a_ref, kl_ref = np.array(alpha_ref_trace), np.array(kl_ref_trace)
    # the schedule keeps every KL well away from Algorithm 1's thresholds 2 kl* and kl* / 2
    for k in kl_ref:
        assert abs(k - 0.02) > 0.1 * 0.02 and abs(k - 0.005) > 0.1 * 0.005, kl_ref
    assert _branches(a_gpu, alpha0) == _branches(a_ref, alpha0), (a_gpu, a_ref)
    assert np.allclose(a_gpu, a_ref, rtol=1e-6, atol=0), (a_gpu, a_ref)
    assert np.allclose(kl_gpu, kl_ref, rtol=1e-4, atol=1e-8), (kl_gpu, kl_ref)
    m, v = L.adam_moments()
    m, v = m.cpu().numpy(), v.cpu().numpy()
    p = L.params().cpu().numpy().astype(np.float64)
    dp, dp_ref = p - flat0, flat_ref - flat0
    ulp = 4 * np.spacing(np.abs(p).astype(np.float32)).astype(np.float64)
    off = 0
    for name, n in _segments(dims):
        sl = slice(off, off + n)
        assert rel_err(m[sl], oracle.m[sl]) < 1e-5, name
        assert rel_err(v[sl], oracle.v[sl]) < 2e-5, name
        assert np.all(np.abs(dp[sl] - dp_ref[sl]) <= 1e-3 * a_ref.sum() + ulp[sl]), name
        off += n


def test_ppo_update_epochs_minibatches_against_oracle():
    """Two rl_ppo_update calls (iterations 0 and 1) against oracle.ppo.update, FP32.  Call 1:
    2 epochs x 2 minibatches from alpha = 1.2e-5 with mean offsets giving KL 0.03 on the first
    minibatch of epoch 0 and 0.001 on the second: alpha / 1.5 clamped at 1e-5, then 1.5 alpha,
    then (epoch 1 mixes both halves, KL ~ 0.0155) alpha unchanged twice.  Call 2: 1 epoch x 2
    minibatches from alpha = 8e-3 with KL 0.001 then 0.03: 1.5 alpha clamped at 1e-2, then
    alpha / 1.5.  Adam runs steps 1-4 and 5-6."""
    w = workload("tiny", epochs=2, minibatches=2)
    L, params, O, Op = _setup(w)
    hidden = w["hidden"]
    B = w["num_envs"] * w["num_steps"]
    dims = (O, hidden, 12)
    rs = np.random.default_rng(99)
    b, d = _batch(B, O, Op, 12, params, hidden, 17, False, kink_margin=True)
    p0 = OM.unflatten(params, O, hidden, 12)
    mu = OM.forward(p0["actor"], b["obs"][:, :O])[0]
    adam = OP.Adam(params.size)
    flat = np.asarray(params, np.float64)
    calls = [(0, 2, 1.2e-5, (0.03, 0.001)), (1, 1, 8e-3, (0.001, 0.03))]
    steps = 0
    for it, epochs, alpha0, kls in calls:
        groups = OP.minibatch_indices(B, 2, w["seed"], it, 0)
        b["mu_old"] = _kl_schedule(mu, p0["log_std"], groups, kls, rs)
        d["mu_old"] = torch.from_numpy(b["mu_old"]).cuda()
        api.rl_set_scalars(L.ctx, alpha0, it, steps)
        stats = torch.empty(api.RL_NSTATS, device="cuda")
        api.rl_ppo_update(L.ctx, d["obs"], d["actions"], d["logp_old"], d["mu_old"], d["v_old"], d["adv"], d["ret"],
                          epochs, 2, 0.2, stats)
        torch.cuda.synchronize()
        batch = {"obs": b["obs"][:, :O], "actions": b["actions"], "logp": b["logp_old"], "mu": b["mu_old"],
                 "values": b["v_old"], "adv": b["adv"], "ret": b["ret"]}
        pcfg = OC.PPOConfig(epochs=epochs, minibatches=2, seed=w["seed"])
        flat_before = flat.copy()
        flat, _, st = OP.update(flat, adam, float(np.float32(alpha0)), batch, O, hidden, 12, pcfg, it)
        steps += epochs * 2
        a_ref = [s["lr"] for s in st]
        kl_ref = [s["kl"] for s in st]
        if it == 0:
            assert _branches(a_ref, alpha0) == ["down", "up", "same", "same"] and a_ref[0] == 1e-5
        else:
            assert _branches(a_ref, alpha0) == ["up", "down"] and a_ref[0] == 1e-2
        sc = api.rl_get_scalars(L.ctx)
        assert sc["adam_step"] == steps and sc["iteration"] == it + 1
        assert abs(float(stats[5].cpu()) - a_ref[-1]) <= 1e-6 * a_ref[-1]
        _check_update(L, adam, flat_before, flat, a_ref, kl_ref, alpha0, dims, len(st))
        # the next call starts from the library's parameters on both sides
        flat = L.params().cpu().numpy().astype(np.float64)
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()


def _bf16_round(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.mark.parametrize("prec,grid,act_ws,fused", [(1, (17, 11), False, False), (0, (17, 11), False, False),
                                                    (1, (12, 9), False, False), (1, (17, 11), True, False),
                                                    (1, (17, 11), False, True)])
def test_train_iteration_rough_teacher_forced(prec, grid, act_ws, fused):
    """One rl_train_iteration of the rough-terrain form: 17 x 11 (or the paper's 108-point 12 x 9)
    height samples, Table 4 noise, pushes, last hidden width 128, so the rollout runs the env step
    with the policy heads fused in (the kernel form the bench times).  The oracle's rollout is
    driven by the library's actions and bootstrap values (teacher forcing); its state then evolves
    bit for bit like the library's: dones, time-outs and levels must match exactly, rewards to
    1e-5, observations within the rounding of their storage type (bf16: half an ulp of the
    oracle's value plus the fp32 path's 1e-5), mu, V, log pi and the sampled actions within the
    precision's tolerance; GAE on the library's rewards and values to 1e-5.  act_ws: the rollout's
    hidden layers in the weight-stationary tile mode, whose launches after the first step fetch
    their weight slice before waiting for the preceding kernel.  fused: the rough task's 512-256-128
    networks with the three hidden layers' forward fused into one launch at both sites."""
    hidden = (512, 256, 128) if fused else (128, 128)
    w = workload("small_rough", precision=prec, grid=grid, crash_threshold=2 ** 26, epochs=1, minibatches=2,
                 hidden=hidden)
    L, params, O, Op = _setup(w)
    if fused:
        api.rl_set_forward_fused(L.ctx, 0, 1)
        api.rl_set_forward_fused(L.ctx, 3, 1)
    if act_ws:
        for layer in range(len(w["hidden"])):
            api.rl_set_gemm_tiles(L.ctx, 3, layer, 64, 5, 1)
    T, N = w["num_steps"], w["num_envs"]
    L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    S = {k: L.storage(i).cpu() for i, k in L.STORAGE.items()}
    S = {k: (v.float() if v.dtype == torch.bfloat16 else v).numpy() for k, v in S.items()}
    hf = synth.heightfield(w["seed"] + 2)
    ol = OLearner(oracle_env_config(w), oracle_ppo_config(w), w["hidden"], hf, params)
    st = ol.rollout(T, actions_override=S["actions"].astype(np.float64),
                    values_override=S["values"].astype(np.float64))
    assert np.array_equal(S["dones"], st["done"]) and np.array_equal(S["timeouts"], st["timeout"])
    assert np.array_equal(S["levels"], st["level"][-1])
    assert S["dones"].sum() > 0
    assert rel_err(S["rewards"], st["reward"]) < TOL_FP32
    obs_gpu, obs_ref = S["obs"][1:T, :, :O], st["obs"][1:]
    assert np.all(S["obs"][:, :, O:] == 0)
    if prec:
        want = _bf16_round(obs_ref)
        scale = np.abs(obs_ref).max()
        assert np.all(np.abs(obs_gpu - want) <= 2 ** -9 * np.abs(want) + TOL_FP32 * scale)
    else:
        assert rel_err(obs_gpu, obs_ref) < TOL_FP32
    tol = TOL_BF16 if prec else TOL_FP32
    for k_gpu, k_ref in (("mu", "mu"), ("values", "values"), ("logp", "logp"), ("actions", "sampled_actions")):
        assert rel_err(S[k_gpu], st[k_ref]) < tol, k_gpu
    assert rel_err(S["last_values"], st["last_values"]) < tol
    A, R = OG.gae(S["rewards"], S["values"], S["last_values"], S["dones"], 0.99, 0.95)
    An, _, _ = OG.normalize(A)
    assert rel_err(S["advantages"], An) < TOL_FP32 and rel_err(S["returns"], R) < TOL_FP32
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()


def test_config_obs_dims_of_the_108_point_grid():
    """The paper's 108 height samples (Sec. 3.2) read as a 12 x 9 grid: 48 + 108 = 156
    observations, padded to 192."""
    w = workload("small_rough", grid=(12, 9))
    assert obs_dims(w) == (156, 192)
    cfg = lib_config(w)
    assert cfg.obs_dim == 156 and cfg.obs_pad == 192


@pytest.mark.parametrize("n,nsplit", [(10007, 1), (16384, 3), (4099, 70)])
def test_adam_step_matches_oracle(n, nsplit):
    """rl_adam_step, the update's Adam kernel on caller buffers: three steps with fresh gradients
    (given as nsplit partial sums; 70 takes the kernel's warp-per-group form, 16384 its 4-wide form),
    against the oracle's Adam (Table 3 betas, bias-corrected, float64 state): moments within 1e-6,
    each step's parameter change within 1e-5 (max-norm relative), and the bf16 copy equal to the new
    parameters rounded to bf16."""
    rng = np.random.default_rng(n + nsplit)
    # parameters of the step's size, so that rounding p to fp32 stays far below the step itself
    p0 = (rng.normal(size=n) * 1e-3).astype(np.float32)
    p = torch.from_numpy(p0).cuda()
    m = torch.zeros(n, device="cuda")
    v = torch.zeros(n, device="cuda")
    wb = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    ad = OP.Adam(n)
    ref = p0.astype(np.float64)
    for t in (1, 2, 3):
        parts = (rng.normal(size=(nsplit, n)) * 0.1).astype(np.float32)
        g = parts.astype(np.float64).sum(0)
        before = p.cpu().numpy().astype(np.float64)
        api.rl_adam_step(p, torch.from_numpy(parts).cuda().reshape(-1), m, v, 1e-3, t, nsplit, wb)
        torch.cuda.synchronize()
        ref_new = ad.step(ref, g, 1e-3)
        got = p.cpu().numpy().astype(np.float64)
        assert rel_err(got - before, ref_new - ref) < 1e-5, t
        assert rel_err(m.cpu().numpy(), ad.m) < 1e-6 and rel_err(v.cpu().numpy(), ad.v) < 1e-6, t
        assert torch.equal(wb.cpu(), p.cpu().to(torch.bfloat16))
        ref = ref_new
    with pytest.raises(api.RLError):
        api.rl_adam_step(p, torch.zeros(n, device="cuda"), m, v, 1e-3, 0)
