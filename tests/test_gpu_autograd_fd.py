"""Central finite differences through the CUDA path: the hand-written backward behind a
torch.autograd.Function (paper_2109_11978_b300.autograd.PPOLoss) against differences of the loss
the library itself evaluates, FP32, on the tiny network with the rough-terrain observation
(O = 235 = 48 + 17 x 11 heights; 64-64 ELU hidden layers).

Every loss evaluation and the gradient run in the library's kernels (rl_set_params +
rl_ppo_loss_grad).  The minibatch keeps every sample away from the kinks of the clipped
surrogate and of the clipped value loss (kink margins far above any step below), so the loss is
smooth inside +-h.

Tolerance (the fp32 cancellation bound): each fp32 loss carries a rounding error of at most
k u |L| (u = 2^-24, k = 16 roundings of the loss's own magnitude along the summation), so the
central difference (L(p + h e) - L(p - h e)) / 2h is off by at most k u |L| / h from the exact
difference quotient; h = 1e-3 keeps the truncation error (h^2 / 6 times the third derivative)
far below that.  Components are tested only where the gradient is at least 20 times that bound.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as OM
from oracle import ppo as OP
from paper_2109_11978_b300 import api
from paper_2109_11978_b300.autograd import ppo_loss
from tests.gpu_helpers import _batch, _segments, _setup
from tests.helpers import TOL_FP32, rel_err, workload

pytestmark = pytest.mark.gpu

H = 1e-3
U = 2.0 ** -24
K_ROUND = 16


def _problem():
    w = workload("tiny", grid=(17, 11))
    L, params, O, Op = _setup(w)
    assert O == 235
    M = w["num_envs"] * w["num_steps"] // w["minibatches"]
    b, d = _batch(M, O, Op, 12, params, w["hidden"], 23, False, kink_margin=True)
    return w, L, params, O, b, d


def test_autograd_function_returns_the_library_gradient():
    """loss.backward() through PPOLoss gives rl_ppo_loss_grad's gradient bit for bit, the loss
    equals the library's statistic, and both match the FP64 oracle to 1e-5."""
    w, L, params, O, b, d = _problem()
    p = torch.from_numpy(params).cuda().requires_grad_()
    loss = ppo_loss(p, L, d)
    loss.backward()
    g_auto = p.grad.clone()
    g_lib = torch.empty(L.n_params, device="cuda")
    stats = torch.empty(api.RL_NSTATS, device="cuda")
    api.rl_ppo_loss_grad(L.ctx, d["obs"], d["actions"], d["logp_old"], d["mu_old"], d["log_std_old"], d["v_old"],
                         d["adv"], d["ret"], g_lib, stats)
    torch.cuda.synchronize()
    assert torch.equal(g_auto, g_lib)
    assert float(loss.detach()) == float(stats[0])
    pr = OM.unflatten(params, O, w["hidden"], 12)
    lref, g, _ = OP.loss_and_grad(pr, b["obs"][:, :O], b["actions"], b["logp_old"], b["mu_old"], b["log_std_old"],
                                  b["v_old"], b["adv"], b["ret"])
    assert abs(float(loss) - lref) <= TOL_FP32 * max(1.0, abs(lref))
    assert rel_err(g_auto.cpu().numpy(), OP.flat_grad(g)) < TOL_FP32
    # a second backward through a scaled loss: the chain-rule factor reaches the gradient
    q = torch.from_numpy(params).cuda().requires_grad_()
    (3.0 * ppo_loss(q, L, d)).backward()
    assert torch.allclose(q.grad, 3.0 * g_lib, rtol=0, atol=0)
    L.close()


def test_central_differences_through_cuda():
    w, L, params, O, b, d = _problem()
    p0 = torch.from_numpy(params).cuda()
    p = p0.clone().requires_grad_()
    loss0 = ppo_loss(p, L, d)
    loss0.backward()
    g = p.grad.cpu().numpy().astype(np.float64)
    Lmag = max(1.0, abs(float(loss0)))
    bound = K_ROUND * U * Lmag / H

    def f(x):
        with torch.no_grad():
            return float(ppo_loss(x, L, d))

    # every tensor of the flat layout: its largest-gradient components and one random one above
    # the threshold
    rs = np.random.default_rng(5)
    checked, off = 0, 0
    worst = 0.0
    for name, n in _segments((O, w["hidden"], 12)):
        seg = np.abs(g[off:off + n])
        ok = np.nonzero(seg >= 20 * bound)[0]
        picks = list(np.argsort(-seg)[:3])
        if ok.size:
            picks.append(int(rs.choice(ok)))
        for i in picks:
            if seg[i] < 20 * bound:
                continue
            e = torch.zeros_like(p0)
            e[off + i] = H
            fd = (f(p0 + e) - f(p0 - e)) / (2 * H)
            err = abs(fd - g[off + i])
            worst = max(worst, err / bound)
            assert err <= bound + 1e-4 * abs(g[off + i]), (name, i, fd, g[off + i], bound)
            checked += 1
        off += n
    assert checked >= 15, checked
    # directional derivatives: along the normalised gradient (d/dt L(p + t u) = |g|) and along two
    # random unit directions over all parameters
    dirs = [g / np.linalg.norm(g)] + [v / np.linalg.norm(v) for v in rs.normal(size=(2, g.size))]
    for u in dirs:
        ut = torch.from_numpy(u.astype(np.float32)).cuda()
        fd = (f(p0 + H * ut) - f(p0 - H * ut)) / (2 * H)
        exact = float(g @ u.astype(np.float32).astype(np.float64))
        assert abs(fd - exact) <= bound + 1e-4 * np.linalg.norm(g), (fd, exact, bound)
    L.close()
