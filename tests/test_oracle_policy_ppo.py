"""Pins of the oracle's policy, PPO loss/gradient, Algorithm 1, Adam and the shuffle (CPU only).

* log-density, entropy and KL of the diagonal Gaussian against scipy's own routines and
  numerical integration; KL(pi, pi) = 0;
* the MLP forward against torch.nn (float64, CPU) as an independent implementation;
* the hand-written gradient of the whole PPO loss against central finite differences (FP64),
  away from the clip kinks, on every parameter of a small network and a sample of the tiny
  configuration's;
* ratio == 1 (parameters equal to the behaviour policy) reduces the surrogate's gradient to
  the vanilla policy gradient -mean(Adv grad log pi) (finite differences of that objective);
* a sample with Adv > 0 and ratio > 1 + clip contributes nothing;
* Algorithm 1 against the hand-worked trace in tests/golden/alg1_trace.txt;
* Adam: first step = -alpha g / (|g| + eps), and 5 steps against torch.optim.Adam;
* the minibatch shuffle is a bijection and matches the scalar Feistel definition.
"""
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.stats

from oracle import config as C
from oracle import mlp, ppo

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_kv(name):
    d = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            d[k] = float(v)
    return d


def test_table3_constants():
    t = _read_kv("table3_ppo.txt")
    assert t["num_robots"] * t["num_steps"] == t["batch_size"]
    assert t["batch_size"] / C.MINIBATCHES == t["minibatch_size"]
    assert (C.EPOCHS, C.CLIP, C.ENTROPY_COEF, C.GAMMA, C.LAM, C.KL_TARGET) == (
        t["epochs"], t["clip"], t["entropy_coef"], t["gamma"], t["lambda"], t["kl_target"])
    assert (C.LR_MIN, C.LR_MAX, C.LR_FACTOR) == (t["lr_min"], t["lr_max"], t["lr_factor"])


def test_gaussian_logprob_entropy_kl():
    rs = np.random.default_rng(0)
    mu, ls, a = rs.normal(size=(5, 12)), rs.normal(0, 0.3, 12), rs.normal(size=(5, 12))
    ref = scipy.stats.norm.logpdf(a, mu, np.exp(ls)).sum(-1)
    np.testing.assert_allclose(mlp.log_prob(a, mu, ls), ref, rtol=1e-12)
    np.testing.assert_allclose(mlp.entropy(ls), scipy.stats.norm.entropy(0, np.exp(ls)).sum(), rtol=1e-12)
    assert abs(mlp.kl_old_new(mu, ls, mu, ls)).max() < 1e-12
    # one dimension against numerical integration of p log(p / q)
    m0, s0, m1, s1 = 0.3, 0.7, -0.2, 1.3
    p = scipy.stats.norm(m0, s0)
    q = scipy.stats.norm(m1, s1)
    num = scipy.integrate.quad(lambda x: p.pdf(x) * (p.logpdf(x) - q.logpdf(x)), -15, 15)[0]
    got = mlp.kl_old_new(np.array([[m0]]), np.log([s0]), np.array([[m1]]), np.log([s1]))[0]
    assert abs(got - num) < 1e-9


def test_mlp_forward_matches_torch():
    torch = pytest.importorskip("torch")
    rs = np.random.default_rng(1)
    dims = [7, 9, 6, 3]
    layers = [(rs.normal(size=(o, i)), rs.normal(size=o)) for i, o in zip(dims[:-1], dims[1:])]
    x = rs.normal(size=(11, 7))
    out, hs = mlp.forward(layers, x)
    mods = []
    for l, (W, b) in enumerate(layers):
        lin = torch.nn.Linear(W.shape[1], W.shape[0]).double()
        lin.weight.data = torch.tensor(W)
        lin.bias.data = torch.tensor(b)
        mods.append(lin)
        if l < len(layers) - 1:
            mods.append(torch.nn.ELU())
    ref = torch.nn.Sequential(*mods)(torch.tensor(x)).detach().numpy()
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)
    z = np.linspace(-3, 3, 61)
    np.testing.assert_allclose(mlp.elu(z), torch.nn.functional.elu(torch.tensor(z)).numpy(), atol=1e-15)
    np.testing.assert_allclose(mlp.elu_grad_from_output(mlp.elu(z)), np.where(z > 0, 1.0, np.exp(z)), atol=1e-15)


def _problem(obs_dim=5, hidden=(6, 4), act_dim=3, M=40, seed=0, offset_ratio=0.0):
    rs = np.random.default_rng(seed)
    n = mlp.param_count(obs_dim, hidden, act_dim)
    flat = rs.normal(0, 0.5, n)
    p = mlp.unflatten(flat, obs_dim, hidden, act_dim)
    obs = rs.normal(size=(M, obs_dim))
    mu, _ = mlp.forward(p["actor"], obs)
    v, _ = mlp.forward(p["critic"], obs)
    a = mu + np.exp(p["log_std"]) * rs.normal(size=mu.shape)
    logp_old = mlp.log_prob(a, mu, p["log_std"]) + offset_ratio * rs.normal(size=M)
    batch = dict(obs=obs, actions=a, logp_old=logp_old, mu_old=mu + 0.05 * rs.normal(size=mu.shape),
                 log_std_old=p["log_std"] + 0.1, v_old=v[:, 0] + 0.3 * rs.normal(size=M),
                 adv=rs.normal(size=M), ret=rs.normal(size=M))
    return flat, batch, (obs_dim, hidden, act_dim)


def _loss(flat, batch, dims, **kw):
    p = mlp.unflatten(flat, *dims)
    return ppo.loss_and_grad(p, batch["obs"], batch["actions"], batch["logp_old"], batch["mu_old"],
                             batch["log_std_old"], batch["v_old"], batch["adv"], batch["ret"], **kw)


def _kink_margin(flat, batch, dims, clip=0.2):
    p = mlp.unflatten(flat, *dims)
    mu, _ = mlp.forward(p["actor"], batch["obs"])
    v, _ = mlp.forward(p["critic"], batch["obs"])
    ratio = np.exp(mlp.log_prob(batch["actions"], mu, p["log_std"]) - batch["logp_old"])
    dv = v[:, 0] - batch["v_old"]
    u = (v[:, 0] - batch["ret"]) ** 2
    w = (batch["v_old"] + np.clip(dv, -clip, clip) - batch["ret"]) ** 2
    out = np.abs(dv) > clip        # inside the clip region w == u identically (no kink)
    uw = np.abs(u - w)[out].min() if out.any() else np.inf
    return min(np.abs(ratio - (1 - clip)).min(), np.abs(ratio - (1 + clip)).min(),
               np.abs(np.abs(dv) - clip).min(), uw)


@pytest.mark.parametrize("offset", [0.0, 0.4])
def test_ppo_gradient_finite_differences_all_params(offset):
    flat, batch, dims = _problem(offset_ratio=offset)
    assert _kink_margin(flat, batch, dims) > 1e-4
    _, grad, _ = _loss(flat, batch, dims)
    g = ppo.flat_grad(grad)
    h = 1e-6
    fd = np.zeros_like(flat)
    for i in range(flat.size):
        e = np.zeros_like(flat)
        e[i] = h
        fd[i] = (_loss(flat + e, batch, dims)[0] - _loss(flat - e, batch, dims)[0]) / (2 * h)
    err = np.abs(fd - g).max() / np.abs(g).max()
    assert err < 1e-7, err


def test_ppo_gradient_finite_differences_tiny_config_sample():
    flat, batch, dims = _problem(obs_dim=48, hidden=(64, 64), act_dim=12, M=64, seed=5, offset_ratio=0.3)
    flat = flat * 0.3
    assert _kink_margin(flat, batch, dims) > 1e-5
    _, grad, _ = _loss(flat, batch, dims)
    g = ppo.flat_grad(grad)
    idx = np.random.default_rng(0).choice(flat.size, 300, replace=False)
    h = 3e-5
    L = abs(_loss(flat, batch, dims)[0])
    roundoff = 8 * np.finfo(np.float64).eps * L / h        # cancellation error of the difference
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (_loss(flat + e, batch, dims)[0] - _loss(flat - e, batch, dims)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * np.abs(g).max() + roundoff, (i, fd, g[i])


def test_ratio_one_reduces_to_vanilla_policy_gradient():
    flat, batch, dims = _problem(M=64, seed=2)
    p = mlp.unflatten(flat, *dims)
    mu, _ = mlp.forward(p["actor"], batch["obs"])
    batch["logp_old"] = mlp.log_prob(batch["actions"], mu, p["log_std"])      # ratio == 1
    _, grad, st = _loss(flat, batch, dims, value_coef=0.0, entropy_coef=0.0)
    g = ppo.flat_grad(grad)
    n_actor = sum(o * i + o for o, i in mlp.layer_dims(dims[0], dims[1], dims[2])) + dims[2]

    def vpg(f):   # -mean(Adv * log pi(a | o; theta)), the vanilla policy-gradient objective
        q = mlp.unflatten(f, *dims)
        m, _ = mlp.forward(q["actor"], batch["obs"])
        return -(batch["adv"] * mlp.log_prob(batch["actions"], m, q["log_std"])).mean()

    h = 1e-6
    for i in range(n_actor):
        e = np.zeros_like(flat)
        e[i] = h
        fd = (vpg(flat + e) - vpg(flat - e)) / (2 * h)
        assert abs(fd - g[i]) < 1e-8 + 1e-7 * np.abs(g).max()
    assert np.all(g[n_actor:] == 0)          # critic untouched when value_coef = 0
    assert abs(st["surrogate"] + batch["adv"].mean()) < 1e-12


def test_clipped_sample_has_no_surrogate_gradient():
    flat, batch, dims = _problem(M=2, seed=4)
    p = mlp.unflatten(flat, *dims)
    mu, _ = mlp.forward(p["actor"], batch["obs"])
    lp = mlp.log_prob(batch["actions"], mu, p["log_std"])
    batch["adv"] = np.array([1.0, 1.0])
    batch["logp_old"] = lp - np.array([0.5, 0.0])          # sample 0: ratio = e^0.5 > 1.2
    _, g_both, _ = _loss(flat, batch, dims, value_coef=0.0, entropy_coef=0.0)
    b1 = {k: (v[1:] if isinstance(v, np.ndarray) and v.ndim and v.shape[0] == 2 else v) for k, v in batch.items()}
    _, g_one, _ = _loss(flat, b1, dims, value_coef=0.0, entropy_coef=0.0)
    # the clipped sample adds nothing; only the 1/M normalisation differs (M = 2 vs 1)
    np.testing.assert_allclose(ppo.flat_grad(g_both) * 2, ppo.flat_grad(g_one), atol=1e-14)


def test_algorithm1_trace():
    lr = 1e-3
    for line in open(os.path.join(GOLD, "alg1_trace.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        kl, want = map(float, line.split())
        lr = ppo.adapt_lr(lr, kl)
        assert abs(lr - want) <= 1e-15 * want, (kl, lr, want)


def test_adam_first_step_and_against_torch():
    torch = pytest.importorskip("torch")
    rs = np.random.default_rng(0)
    p0, g = rs.normal(size=50), rs.normal(size=50)
    ad = ppo.Adam(50)
    p1 = ad.step(p0, g, 1e-3)
    np.testing.assert_allclose(p1, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    tp = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    ad = ppo.Adam(50)
    p = p0.copy()
    for k in range(5):
        gk = rs.normal(size=50)
        lr = 1e-3 * (1 + k)
        for grp in opt.param_groups:
            grp["lr"] = lr
        tp.grad = torch.tensor(gk)
        opt.step()
        p = ad.step(p, gk, lr)
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 768, 1000, 4096, 98304])
def test_permutation_bijective(n):
    k = 0xDEADBEEF12345678
    perm = ppo.permutation(n, k)
    assert np.array_equal(np.sort(perm), np.arange(n))
    if n <= 1000:
        half = ppo.feistel_bits(n) // 2
        for i in range(n):
            y = ppo.feistel(i, k, half)
            while y >= n:
                y = ppo.feistel(y, k, half)
            assert y == perm[i]


def test_minibatches_partition_batch():
    mbs = ppo.minibatch_indices(96, 4, 3, 1, 2)
    assert len(mbs) == 4 and all(len(m) == 24 for m in mbs)
    assert np.array_equal(np.sort(np.concatenate(mbs)), np.arange(96))
    other = ppo.minibatch_indices(96, 4, 3, 1, 3)
    assert not np.array_equal(np.concatenate(mbs), np.concatenate(other))


def test_loss_and_grad_hand_worked_example():
    """oracle.ppo.loss_and_grad on the three-sample example worked by hand in
    tests/golden/ppo_loss_hand.txt: each branch of the clipped surrogate and of the clipped value
    loss, the entropy bonus with its sign and weight, and the composed loss and head gradients."""
    t = _read_kv("ppo_loss_hand.txt")
    O, hidden, A = 2, (4,), 12
    p = mlp.unflatten(np.zeros(mlp.param_count(O, hidden, A)), O, hidden, A)
    p["critic"][-1] = (p["critic"][-1][0], np.array([0.5]))
    obs = np.array([[0.3, -1.0], [2.0, 0.5], [-0.7, 0.1]])
    actions = np.full((3, A), 0.5)
    logp = mlp.log_prob(actions, np.zeros((3, A)), p["log_std"])
    assert np.allclose(logp, t["logp"], rtol=0, atol=1e-12)
    logp_old = logp - np.array([0.0, 0.5, -0.5])
    adv = np.array([1.0, 2.0, 1.0])
    v_old = np.array([0.5, 0.0, 0.0])
    ret = np.array([1.5, 1.0, 0.0])
    loss, g, st = ppo.loss_and_grad(p, obs, actions, logp_old, np.zeros((3, A)), np.zeros(A), v_old, adv, ret)
    for k in ("surrogate", "value_loss", "entropy", "loss", "clip_frac", "kl"):
        assert abs(st[k] - t[k]) <= 1e-12 * max(1.0, abs(t[k])), (k, st[k], t[k])
    assert abs(loss - t["loss"]) <= 1e-12
    assert np.allclose(g["actor"][-1][1], t["grad_actor_bias"], rtol=0, atol=1e-12)
    assert np.allclose(g["log_std"], t["grad_log_std"], rtol=0, atol=1e-12)
    assert np.allclose(g["critic"][-1][1], t["grad_critic_bias"], rtol=0, atol=1e-12)
    for net in ("actor", "critic"):
        for l, (gw, gb) in enumerate(g[net]):
            assert not np.any(gw), (net, l)
            if l < len(g[net]) - 1:
                assert not np.any(gb), (net, l)
