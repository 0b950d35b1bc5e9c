"""GPU parity (through the C ABI) of policy inference, the PPO loss/gradient, the update and a
whole training iteration against the FP64 oracle.

FP32 form: 1e-5 relative (|x - ref|_inf / |ref|_inf per tensor) for mu, V, log pi, actions, loss
terms and every gradient tensor.  BF16 form (bf16 GEMM operands, FP32 accumulation): 2e-2 in the
same max-norm, for the forward outputs and for every gradient tensor (on a minibatch kept away from
the clip kinks, where only rounding separates the two paths).
Adam after one step is -alpha g / (|g| + eps), i.e. alpha times the sign of g for all but the
smallest gradients: elements whose oracle gradient exceeds 1e-3 of the tensor's largest must
match to 1e-5 alpha, every other element must stay within the step bound alpha.
"""
import numpy as np
import pytest
import torch

from oracle import gae as OG
from oracle import mlp as OM
from oracle import ppo as OP
from oracle.train import Learner as OLearner
from paper_2109_11978_b300 import api
from tests.gpu_helpers import _batch, _obs, _own_old_policy, _per_tensor_err, _segments, _setup
from tests.helpers import TOL_BF16, TOL_FP32, oracle_env_config, oracle_ppo_config, rel_err, workload

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,form,rows", [("tiny", "fp32", 64), ("rough", "fp32", 4096), ("tiny", "bf16", 64),
                                            ("rough", "bf16", 4096), ("rough", "bf16", 1000)])
def test_policy_act(name, form, rows):
    prec = 1 if form == "bf16" else 0
    w = workload(name, precision=prec)
    L, params, O, Op = _setup(w)
    x, xd = _obs(rows, O, Op, 3, prec == 1)
    act = torch.empty((rows, 12), device="cuda")
    mu = torch.empty((rows, 12), device="cuda")
    lp = torch.empty(rows, device="cuda")
    v = torch.empty(rows, device="cuda")
    api.rl_policy_act(L.ctx, 3, xd, act, mu, lp, v)
    v2 = torch.empty(rows, device="cuda")
    api.rl_policy_act(L.ctx, 3, xd, None, None, None, v2)
    torch.cuda.synchronize()
    p = OM.unflatten(params, O, w["hidden"], 12)
    ref = OM.act(p, x[:, :O], w["seed"], 0, 3)
    tol = TOL_FP32 if prec == 0 else TOL_BF16
    for k, got in (("mu", mu), ("values", v), ("actions", act), ("logp", lp)):
        assert rel_err(got.cpu().numpy(), ref[k]) < tol, k
    assert torch.equal(v, v2)
    L.close()


@pytest.mark.parametrize("name,form,hidden", [("tiny", "fp32", None), ("rough", "fp32", None), ("tiny", "bf16", None),
                                              ("rough", "bf16", None), ("tiny", "bf16", (128, 256)),
                                              ("tiny", "fp32", (128, 256))])
def test_ppo_loss_grad(name, form, hidden):
    """FP32: the oracle and the GPU get identical inputs.  BF16: as in training, log pi_old, V_old
    and mu_old come from each path's own inference at the same parameters (plus identical offsets),
    so the bf16 forward error cancels inside the ratio exactly as it does in the loop; the batch is
    kept away from the clip kinks.  A last hidden layer of 256 runs the loss head's tensor-core
    form, 64 and 128 its warp-per-row form."""
    prec = 1 if form == "bf16" else 0
    w = workload(name, precision=prec, **({"hidden": hidden} if hidden else {}))
    L, params, O, Op = _setup(w)
    M = w["num_envs"] * w["num_steps"] // w["minibatches"]
    b, d = _batch(M, O, Op, 12, params, w["hidden"], 21, prec == 1, kink_margin=prec == 1)
    if prec == 1:
        d = _own_old_policy(L, b, d, O, params, w["hidden"])
    grad = torch.empty(L.n_params, device="cuda")
    stats = torch.empty(16, device="cuda")
    api.rl_ppo_loss_grad(L.ctx, d["obs"], d["actions"], d["logp_old"], d["mu_old"], d["log_std_old"], d["v_old"],
                         d["adv"], d["ret"], grad, stats)
    torch.cuda.synchronize()
    p = OM.unflatten(params, O, w["hidden"], 12)
    _, g, st = OP.loss_and_grad(p, b["obs"][:, :O], b["actions"], b["logp_old"], b["mu_old"], b["log_std_old"],
                                b["v_old"], b["adv"], b["ret"])
    gref = OP.flat_grad(g)
    tol = TOL_FP32 if prec == 0 else TOL_BF16
    errs = _per_tensor_err(grad.cpu().numpy(), gref, (O, w["hidden"], 12), rel_err)
    bad = {k: e for k, e in errs.items() if e >= tol}
    assert not bad, (bad, errs)
    s = stats.cpu().numpy()
    for i, k in ((0, "loss"), (1, "surrogate"), (2, "value_loss"), (3, "entropy")):
        assert abs(s[i] - st[k]) <= tol * max(1.0, abs(st[k])), (k, s[i], st[k])
    assert abs(s[4] - st["kl"]) <= tol * max(st["kl"], 1e-3)
    assert 0.05 < st["clip_frac"] < 0.95
    L.close()


def test_ppo_single_step_adam_and_alg1():
    w = workload("tiny", epochs=1, minibatches=1)
    L, params, O, Op = _setup(w)
    B = w["num_envs"] * w["num_steps"]
    b, d = _batch(B, O, Op, 12, params, w["hidden"], 5, False)
    b["mu_old"][:] = OM.forward(OM.unflatten(params, O, w["hidden"], 12)["actor"], b["obs"][:, :O])[0]
    d["mu_old"] = torch.from_numpy(b["mu_old"]).cuda()
    api.rl_ppo_update(L.ctx, d["obs"], d["actions"], d["logp_old"], d["mu_old"], d["v_old"], d["adv"], d["ret"], 1, 1, 0.2)
    newp = L.params().cpu().numpy().astype(np.float64)
    sc = api.rl_get_scalars(L.ctx)
    assert sc["iteration"] == 1 and sc["adam_step"] == 1
    assert sc["alpha"] == np.float32(np.float32(1e-3) * np.float32(1.5))    # KL ~ 0 < kl*/2 -> alpha * 1.5
    p = OM.unflatten(params, O, w["hidden"], 12)
    log_std_old = p["log_std"].copy()
    _, g, _ = OP.loss_and_grad(p, b["obs"][:, :O], b["actions"], b["logp_old"], b["mu_old"], log_std_old, b["v_old"],
                               b["adv"], b["ret"])
    gref = OP.flat_grad(g)
    alpha = float(sc["alpha"])
    dref = -alpha * gref / (np.abs(gref) + 1e-8)
    dgot = newp - params.astype(np.float64)
    ulp = 2 * np.spacing(np.abs(params).astype(np.float32)).astype(np.float64)   # fp32 rounding of p + dp
    off = 0
    for name, n in _segments((O, w["hidden"], 12)):
        gs, dr, dg, u = gref[off:off + n], dref[off:off + n], dgot[off:off + n], ulp[off:off + n]
        firm = np.abs(gs) > 1e-3 * np.abs(gs).max()
        assert np.all(np.abs(dg[firm] - dr[firm]) <= TOL_FP32 * alpha + u[firm]), name
        assert np.all(np.abs(dg) <= alpha * (1 + 1e-5) + u), name
        off += n
    L.close()


def test_train_iteration_against_oracle_teacher_forced():
    w = workload("tiny", epochs=2, minibatches=2, crash_threshold=2 ** 26)
    L, params, O, Op = _setup(w)
    ecfg, pcfg = oracle_env_config(w), oracle_ppo_config(w)
    T, N = w["num_steps"], w["num_envs"]
    L.train_iteration(use_graph=False)
    torch.cuda.synchronize()
    S = {k: L.storage(i).cpu().numpy() for i, k in L.STORAGE.items()}
    ol = OLearner(ecfg, pcfg, w["hidden"], np.zeros((800, 1600), np.float32), params)
    st = ol.rollout(T, actions_override=S["actions"].astype(np.float64))
    # obs[t] for t >= 1 came from env step t - 1; obs[0] already holds the next iteration's first
    # observation (copied from obs[T] at the end of the iteration)
    assert rel_err(S["obs"][1:T, :, :O], st["obs"][1:]) < TOL_FP32
    assert rel_err(S["obs"][0, :, :O], ol.obs) < TOL_FP32 and rel_err(S["obs"][T, :, :O], ol.obs) < TOL_FP32
    assert rel_err(S["rewards"], st["reward"]) < TOL_FP32
    assert np.array_equal(S["dones"], st["done"]) and np.array_equal(S["timeouts"], st["timeout"])
    assert np.array_equal(S["levels"], st["level"][-1])
    assert S["dones"].sum() > 0
    for k_gpu, k_ref in (("mu", "mu"), ("values", "values"), ("logp", "logp")):
        assert rel_err(S[k_gpu], st[k_ref]) < TOL_FP32, k_gpu
    assert rel_err(S["last_values"], st["last_values"]) < TOL_FP32
    # GAE on the GPU's rewards and values
    A, R = OG.gae(S["rewards"], S["values"], S["last_values"], S["dones"], pcfg.gamma, pcfg.lam)
    An, _, _ = OG.normalize(A)
    assert rel_err(S["advantages"], An) < TOL_FP32 and rel_err(S["returns"], R) < TOL_FP32
    # iteration counter, stats
    sc = api.rl_get_scalars(L.ctx)
    assert sc["iteration"] == 1 and sc["adam_step"] == pcfg.epochs * pcfg.minibatches
    stats = S["stats"]
    assert abs(stats[7] - S["rewards"].mean()) < 1e-5 * max(1.0, abs(S["rewards"].mean()))
    assert stats[10] == S["dones"].sum()
    L.close()


def test_graph_replay_equals_eager():
    w = workload("tiny", epochs=2, minibatches=2)
    La, params, O, Op = _setup(w)
    Lb, _, _, _ = _setup(w)
    for _ in range(2):
        La.train_iteration(use_graph=True)
        Lb.train_iteration(use_graph=False)
    torch.cuda.synchronize()
    assert torch.equal(La.params(), Lb.params())
    for i in (0, 1, 5, 6, 9):
        assert torch.equal(La.storage(i), Lb.storage(i)), i
    assert api.rl_last_device_status(La.ctx) == 0
    La.close()
    Lb.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_side_streams_equal_serial_order(prec):
    """With per-class profiling every launch of the iteration stays on the main stream; without it
    the shuffle, the record packing, the next minibatch's gather and the weight gradients run on
    side streams.  Both orders give the same bits."""
    w = workload("tiny", precision=prec, epochs=2, minibatches=2)
    La, _, _, _ = _setup(w)
    Lb, _, _, _ = _setup(w)
    api.rl_profile_enable(Lb.ctx, api.RL_PROF_ALL, True)
    for _ in range(2):
        La.train_iteration(use_graph=True)
        Lb.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    assert torch.equal(La.params(), Lb.params())
    for i in (0, 1, 5, 6, 9):
        assert torch.equal(La.storage(i), Lb.storage(i)), i
    assert api.rl_get_scalars(La.ctx) == api.rl_get_scalars(Lb.ctx)
    assert api.rl_last_device_status(La.ctx) == 0 and api.rl_last_device_status(Lb.ctx) == 0
    La.close()
    Lb.close()


@pytest.mark.parametrize("form", ["fp32", "bf16"])
def test_autotune_keeps_results(form):
    """The autotuner only changes tile widths and split counts: the gradient stays within the
    tolerance of the oracle, and the report names every GEMM site it timed."""
    prec = 1 if form == "bf16" else 0
    w = workload("tiny", precision=prec)
    L, params, O, Op = _setup(w)
    M = w["num_envs"] * w["num_steps"] // w["minibatches"]
    b, d = _batch(M, O, Op, 12, params, w["hidden"], 31, prec == 1, kink_margin=prec == 1)
    if prec == 1:
        d = _own_old_policy(L, b, d, O, params, w["hidden"])

    def grad():
        g = torch.empty(L.n_params, device="cuda")
        api.rl_ppo_loss_grad(L.ctx, d["obs"], d["actions"], d["logp_old"], d["mu_old"], d["log_std_old"], d["v_old"],
                             d["adv"], d["ret"], g)
        torch.cuda.synchronize()
        return g.cpu().numpy()

    g0 = grad()
    rep = api.rl_autotune(L.ctx)
    sites = {(s["site"], s["layer"]) for s in rep["sites"]}
    assert ("weight_grad", 0) in sites and ("weight_grad", len(w["hidden"]) - 1) in sites
    if prec == 1:
        assert ("forward", 0) in sites and ("input_grad", 1) in sites
    g1 = grad()
    p = OM.unflatten(params, O, w["hidden"], 12)
    _, g, _ = OP.loss_and_grad(p, b["obs"][:, :O], b["actions"], b["logp_old"], b["mu_old"], b["log_std_old"],
                               b["v_old"], b["adv"], b["ret"])
    gref = OP.flat_grad(g)
    tol = TOL_FP32 if prec == 0 else TOL_BF16
    for gg in (g0, g1):
        errs = _per_tensor_err(gg, gref, (O, w["hidden"], 12), rel_err)
        assert max(errs.values()) < tol, errs
    L.train_iteration(use_graph=True)          # the graph is re-captured with the tuned shapes
    torch.cuda.synchronize()
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()


@pytest.mark.parametrize("bn,cm,splits", [(64, 1, "one"), (64, 1, "most"), (128, 1, "most"), (128, 1, "one"),
                                          (256, 1, "one"), (256, 1, "most"), (128, 3, "one"), (256, 3, "most"),
                                          (64, 4, "most"), (128, 4, "one"), (128, 4, "most"), (64, 5, "one"),
                                          (128, 5, "one"), (256, 5, "one")])
def test_gemm_tile_shapes_keep_results(bn, cm, splits):
    """Every tile width and tile mode of the tensor-core GEMM (1: one CTA per tile; 3: CTA pairs
    on the cta_group::2 MMA; 4: two K blocks per pipeline stage, so splits of an odd K-block count
    end on a half-used stage; 5: weight-stationary, the forward and input-gradient sites only, with
    more CTAs per (network, column tile) group than the rollout site's 4 row tiles, so some CTAs
    have no tile), pinned at every site where it is valid, gives
    the oracle's gradient within the BF16 tolerance.  2880 minibatch rows = 23 row tiles: the last
    pair of a cluster has one tile past the rows, and the last row tile is ragged."""
    w = workload("rough", num_envs=480, precision=1)
    L, params, O, Op = _setup(w)
    M = w["num_envs"] * w["num_steps"] // w["minibatches"]
    assert M == 2880
    hidden = w["hidden"]
    widths = {0: hidden, 1: [Op] + list(hidden[:-1])}     # output width of forward / input-gradient sites
    pinned = 0
    for layer in range(len(hidden)):
        for site in (0, 1, 2, 3):
            if site == 1 and layer == 0:
                continue
            width = hidden[layer] if site in (0, 3) else widths[1][layer]
            out_tiles = -(-hidden[layer] // 128)
            paired = cm == 3
            if (width % bn or (site == 2 and paired and out_tiles < 2) or (paired and bn < 128 and (cm == 3 or site in (1, 2)))
                    or (cm == 4 and bn > 128)):
                continue
            choices = [1] if splits == "one" else [64, 48, 32, 24, 16, 12, 8, 6, 4, 3, 2]
            for s_ in choices:
                try:
                    api.rl_set_gemm_tiles(L.ctx, site, layer, bn, cm, s_)
                    pinned += 1
                    break
                except api.RLError:
                    continue
    assert pinned >= 3
    b, d = _batch(M, O, Op, 12, params, hidden, 41, True, kink_margin=True)
    d = _own_old_policy(L, b, d, O, params, hidden)
    g = torch.empty(L.n_params, device="cuda")
    api.rl_ppo_loss_grad(L.ctx, d["obs"], d["actions"], d["logp_old"], d["mu_old"], d["log_std_old"], d["v_old"],
                         d["adv"], d["ret"], g)
    torch.cuda.synchronize()
    assert api.rl_last_device_status(L.ctx) == 0
    p = OM.unflatten(params, O, hidden, 12)
    _, gr, _ = OP.loss_and_grad(p, b["obs"][:, :O], b["actions"], b["logp_old"], b["mu_old"], b["log_std_old"],
                                b["v_old"], b["adv"], b["ret"])
    errs = _per_tensor_err(g.cpu().numpy(), OP.flat_grad(gr), (O, hidden, 12), rel_err)
    assert max(errs.values()) < TOL_BF16, errs
    L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()


def test_set_gemm_tiles_rejects_invalid():
    w = workload("tiny", precision=1)
    L, _, _, _ = _setup(w)
    # (site, layer, bn, cluster, splits): the weight-stationary mode 5 is refused at the weight
    # gradient, the split-reducing modes 6 and 7 everywhere else, mode 7 above a tile width of 128;
    # mode 8 does not exist
    for args in ((4, 0, 64, 1, 1), (1, 0, 64, 1, 1), (0, 0, 96, 1, 1), (0, 0, 64, 6, 1), (0, 9, 64, 1, 1),
                 (2, 0, 64, 1, 0), (3, 0, 128, 1, 1), (0, 0, 64, 3, 1), (0, 0, 256, 4, 1), (0, 0, 64, 2, 1),
                 (0, 0, 128, 2, 1), (2, 0, 64, 5, 1), (3, 0, 64, 7, 1), (2, 0, 256, 7, 2), (0, 0, 64, 8, 1)):
        with pytest.raises(api.RLError):
            api.rl_set_gemm_tiles(L.ctx, *args)
    L.close()


def test_profile_classes_count_every_launch():
    """In-graph timing by kernel class: one event pair per launch, counted per class, with the
    launch counts the iteration's structure fixes (T env steps, each with the rollout's policy head
    fused in, one action-head pass for the bootstrap value, epochs x minibatches loss heads,
    gathers and Adam steps)."""
    w = workload("tiny", precision=1)
    L, _, _, _ = _setup(w)
    api.rl_profile_enable(L.ctx, api.RL_PROF_ALL, True)
    L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    n_mb = w["epochs"] * w["minibatches"]
    counts = {name: api.rl_profile_read_class(L.ctx, i)[1] for i, name in enumerate(api.RL_PROF_NAMES)}
    assert counts["env_step"] == w["num_steps"]
    assert counts["act_head"] == 1
    # the loss head and its statistics / Algorithm 1 kernel per minibatch
    assert counts["loss_head"] == 2 * n_mb and counts["adam"] == n_mb and counts["gather"] == n_mb
    nh = len(w["hidden"])
    assert counts["gemm"] == (w["num_steps"] + 1) * nh + n_mb * (3 * nh - 1)
    total_ms, total_n = api.rl_profile_read(L.ctx)
    assert total_n == sum(counts.values()) and total_ms > 0
    with pytest.raises(api.RLError):
        api.rl_profile_read_class(L.ctx, api.RL_PROF_ALL)
    api.rl_profile_enable(L.ctx, api.RL_PROF_ALL, False)
    L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    assert api.rl_profile_read(L.ctx)[1] == 0
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()


@pytest.mark.parametrize("splits,bn,cm", [(8, 128, 6), (12, 128, 7), (6, 64, 6), (9, 128, 7)])
def test_weight_gradient_split_reduction_in_clusters(splits, bn, cm):
    """Tile modes 6 and 7 of the weight gradient: the split-K partials reduced inside the GEMM by
    clusters of CTAs (the largest divisor of the split count up to 8: 8, 6, 6 and 3 here), Adam
    summing the clusters' partials, give the gradient of the plain modes 1 and 4 to fp32 rounding and
    the oracle's gradient within the BF16 tolerance; 2880 minibatch rows with splits of whole 64-row
    blocks (the last split of 8 and 12 ragged)."""
    w = workload("rough", num_envs=480, precision=1)
    L, params, O, Op = _setup(w)
    M = w["num_envs"] * w["num_steps"] // w["minibatches"]
    hidden = w["hidden"]
    b, d = _batch(M, O, Op, 12, params, hidden, 43, True, kink_margin=True)
    d = _own_old_policy(L, b, d, O, params, hidden)
    grads = {}
    plain = {6: 1, 7: 4}[cm]
    for mode in (cm, plain):
        for layer in range(len(hidden)):
            api.rl_set_gemm_tiles(L.ctx, 2, layer, bn, mode, splits)
        g = torch.empty(L.n_params, device="cuda")
        api.rl_ppo_loss_grad(L.ctx, d["obs"], d["actions"], d["logp_old"], d["mu_old"], d["log_std_old"], d["v_old"],
                             d["adv"], d["ret"], g)
        torch.cuda.synchronize()
        assert api.rl_last_device_status(L.ctx) == 0
        grads[mode] = g.cpu().numpy().astype(np.float64)
    scale = np.abs(grads[plain]).max()
    assert np.abs(grads[cm] - grads[plain]).max() <= 1e-5 * scale
    p = OM.unflatten(params, O, hidden, 12)
    _, gr, _ = OP.loss_and_grad(p, b["obs"][:, :O], b["actions"], b["logp_old"], b["mu_old"], b["log_std_old"],
                                b["v_old"], b["adv"], b["ret"])
    errs = _per_tensor_err(grads[cm], OP.flat_grad(gr), (O, hidden, 12), rel_err)
    assert max(errs.values()) < TOL_BF16, errs
    for layer in range(len(hidden)):
        api.rl_set_gemm_tiles(L.ctx, 2, layer, bn, cm, splits)
    with pytest.raises(api.RLError):
        api.rl_set_gemm_tiles(L.ctx, 0, 0, 128, 6, 1)          # modes 6, 7: weight gradients only
    L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()
