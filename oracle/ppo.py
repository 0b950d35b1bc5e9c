"""PPO update with clipped surrogate, adaptive-KL learning rate and Adam (oracle, FP64).

Test infrastructure only.  Follows:
* Sec. 2.2 and Table 3: PPO (Schulman et al. 2017) with clip range 0.2, entropy
  coefficient 0.01, 5 epochs, 4 minibatches of B/4 = 24576 samples, gamma 0.99, lambda 0.95;
* Algorithm 1 (App. A.4): after each minibatch forward pass, kl = KL between the old and
  the new policy; alpha <- max(1e-5, alpha / 1.5) if kl > 2 kl*, alpha <- min(1e-2, 1.5 alpha)
  if kl < kl* / 2, kl* = 0.01;
* the clipped value loss (value coefficient 1), the minibatch shuffle per epoch, the KL
  direction KL(pi_old || pi_new) and Adam with PyTorch's default betas/eps are the readings
  this build takes where the paper is silent.

Per sample i of a minibatch of size M (A = action dims):
    ratio_i = exp(log pi(a_i) - log pi_old(a_i))
    L_surr  = -(1/M) sum_i min(ratio_i Adv_i, clip(ratio_i, 1 - c, 1 + c) Adv_i)
    V_clip  = V_old + clip(V - V_old, -c, c)
    L_V     = (1/M) sum_i max((V_i - R_i)^2, (V_clip,i - R_i)^2)
    H       = sum_j (log sigma_j + 0.5 log(2 pi e))
    loss    = L_surr + value_coef L_V - entropy_coef H
The gradient is derived by hand (chain rule through the heads, the ELU layers and the
linear layers) and pinned against central finite differences in tests.
"""
import numpy as np

from . import mlp, rng


def loss_and_grad(p, obs, actions, logp_old, mu_old, log_std_old, v_old, adv, ret,
                  clip=0.2, value_coef=1.0, entropy_coef=0.01):
    obs = np.asarray(obs, np.float64)
    actions = np.asarray(actions, np.float64)
    M = obs.shape[0]
    mu, hs_a = mlp.forward(p["actor"], obs)
    v, hs_c = mlp.forward(p["critic"], obs)
    v = v[:, 0]
    ls = p["log_std"]
    var = np.exp(2.0 * ls)
    logp = mlp.log_prob(actions, mu, ls)
    ratio = np.exp(logp - logp_old)
    s1 = ratio * adv
    s2 = np.clip(ratio, 1.0 - clip, 1.0 + clip) * adv
    surr = -np.minimum(s1, s2).mean()
    dv = v - v_old
    v_clip = v_old + np.clip(dv, -clip, clip)
    u = (v - ret) ** 2
    w = (v_clip - ret) ** 2
    vloss = np.maximum(u, w).mean()
    ent = mlp.entropy(ls)
    loss = surr + value_coef * vloss - entropy_coef * ent
    kl = mlp.kl_old_new(mu_old, log_std_old, mu, ls).mean()

    # d loss / d ratio: the unclipped branch carries the gradient when it is the minimum.
    g_ratio = -np.where(s1 <= s2, adv, 0.0) / M
    g_logp = g_ratio * ratio
    diff = actions - mu
    g_mu = g_logp[:, None] * diff / var
    g_ls = (g_logp[:, None] * (diff ** 2 / var - 1.0)).sum(0) - entropy_coef
    inside = (dv > -clip) & (dv < clip)
    g_v = value_coef / M * np.where(u >= w, 2.0 * (v - ret), 2.0 * (v_clip - ret) * inside)

    ga = backward(p["actor"], hs_a, g_mu)
    gc = backward(p["critic"], hs_c, g_v[:, None])
    grad = {"actor": ga, "critic": gc, "log_std": g_ls}
    stats = {"loss": loss, "surrogate": surr, "value_loss": vloss, "entropy": ent, "kl": kl,
             "clip_frac": float((np.abs(ratio - 1.0) > clip).mean())}
    return loss, grad, stats


def loss_only(p, *args, **kw):
    return loss_and_grad(p, *args, **kw)[0]


def backward(layers, hs, g_out):
    """Gradients of every (W, b) given d loss / d output; hs[l] is layer l's input."""
    grads = [None] * len(layers)
    g = g_out
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (g.T @ hs[l], g.sum(0))
        if l > 0:
            g = (g @ W) * mlp.elu_grad_from_output(hs[l])
    return grads


def adapt_lr(lr, kl, kl_target=0.01, lr_min=1e-5, lr_max=1e-2, factor=1.5):
    """Algorithm 1 (App. A.4)."""
    if kl > 2.0 * kl_target:
        return max(lr_min, lr / factor)
    if kl < 0.5 * kl_target:
        return min(lr_max, lr * factor)
    return lr


class Adam:
    """Adam (Kingma & Ba 2015, Algorithm 1) with bias correction, float64 state."""

    def __init__(self, n, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.step_count = 0
        self.b1, self.b2, self.eps = beta1, beta2, eps

    def step(self, params, grad, lr):
        self.step_count += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * grad
        self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
        mhat = self.m / (1.0 - self.b1 ** self.step_count)
        vhat = self.v / (1.0 - self.b2 ** self.step_count)
        return params - lr * mhat / (np.sqrt(vhat) + self.eps)


def feistel_bits(n):
    """Even bit width 2h with 2^(2h) >= n (at least 2)."""
    b = 2
    while (1 << b) < n:
        b += 2
    return b


def feistel(x, k, half):
    """4-round balanced Feistel network on 2*half-bit integers, round function from mix64."""
    mask = (1 << half) - 1
    L, R = x >> half, x & mask
    for r in range(4):
        F = rng.mix64((k + ((r + 1) << 32) + R) & rng.MASK) & mask
        L, R = R, L ^ F
    return (L << half) | R


def permutation(n, k):
    """Permutation of range(n) by cycle-walking the Feistel network (bijective by construction).

    Vectorised over all n inputs (numpy uint64, wrapping arithmetic); same function as the
    scalar feistel() above, which the tests use as the brute-force check.
    """
    half = feistel_bits(n) // 2
    mask = np.uint64((1 << half) - 1)
    kk = np.uint64(k)

    def f(x):
        L, R = x >> np.uint64(half), x & mask
        for r in range(4):
            F = rng.mix64(kk + np.uint64((r + 1) << 32) + R) & mask
            L, R = R, L ^ F
        return (L << np.uint64(half)) | R

    y = f(np.arange(n, dtype=np.uint64))
    while True:
        bad = y >= np.uint64(n)
        if not bad.any():
            return y.astype(np.int64)
        y[bad] = f(y[bad])


def minibatch_indices(n, minibatches, seed, iteration, epoch):
    k = int(rng.key(seed, rng.STREAM_PERM, iteration, epoch, 0))
    perm = permutation(n, k)
    mb = n // minibatches
    return [perm[m * mb:(m + 1) * mb] for m in range(minibatches)]


def flat_grad(grad):
    return mlp.flatten({"actor": grad["actor"], "log_std": grad["log_std"], "critic": grad["critic"]})


def update(flat, adam, lr, batch, obs_dim, hidden, act_dim, cfg, iteration):
    """All epochs x minibatches of one iteration.  batch: dict of [B, ...] arrays with keys
    obs, actions, logp, mu, values, adv (normalised), ret.  Returns (flat, lr, stats list)."""
    flat = np.asarray(flat, np.float64).copy()
    B = batch["obs"].shape[0]
    log_std_old = mlp.unflatten(flat, obs_dim, hidden, act_dim)["log_std"].copy()
    stats = []
    for e in range(cfg.epochs):
        for idx in minibatch_indices(B, cfg.minibatches, cfg.seed, iteration, e):
            p = mlp.unflatten(flat, obs_dim, hidden, act_dim)
            _, grad, st = loss_and_grad(
                p, batch["obs"][idx], batch["actions"][idx], batch["logp"][idx],
                batch["mu"][idx], log_std_old, batch["values"][idx], batch["adv"][idx],
                batch["ret"][idx], cfg.clip, cfg.value_coef, cfg.entropy_coef)
            lr = adapt_lr(lr, st["kl"], cfg.kl_target, cfg.lr_min, cfg.lr_max)
            flat = adam.step(flat, flat_grad(grad), lr)
            st["lr"] = lr
            stats.append(st)
    return flat, lr, stats
