"""Helpers of the GPU tests: learners built from the named workloads, seeded minibatches for the
PPO loss, the old-policy quantities each path produces, and per-tensor error measures over the flat
parameter layout."""
import numpy as np
import torch

from oracle import mlp as OM
from paper_2109_11978_b300 import api, synth
from tests.helpers import lib_config, obs_dims, rel_err


def _bf16(x):
    return torch.as_tensor(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy()


def _setup(w):
    cfg = lib_config(w)
    O, Op = obs_dims(w)
    params = synth.xavier_params(w["seed"] + 1, O, w["hidden"], 12, log_std=-0.3, bias_scale=0.1)
    hf = synth.heightfield(w["seed"] + 2) if w["grid"][0] else None
    return api.Learner(cfg, hf, params), params, O, Op


def _obs(rows, O, Op, seed, bf16):
    x = np.zeros((rows, Op), np.float32)
    x[:, :O] = np.random.default_rng(seed).normal(size=(rows, O))
    if bf16:
        x = _bf16(x)
        return x, torch.from_numpy(x).to(torch.bfloat16).cuda()
    return x, torch.from_numpy(x).cuda()


def _segments(dims):
    """(name, size) of every tensor in the flat layout."""
    O, hidden, A = dims
    out = []
    for net, od in (("actor", A), ("critic", 1)):
        for l, (o, i) in enumerate(OM.layer_dims(O, hidden, od)):
            out += [(f"{net}.W{l}", o * i), (f"{net}.b{l}", o)]
        if net == "actor":
            out.append(("log_std", A))
    return out


def _per_tensor_err(g, ref, dims, measure=rel_err):
    errs, off = {}, 0
    for name, n in _segments(dims):
        errs[name] = measure(g[off:off + n], ref[off:off + n])
        off += n
    return errs


def _batch(M, O, Op, A, params, hidden, seed, bf16, kink_margin=False):
    """A minibatch whose ratios straddle the clip range and whose values straddle the value clip.

    kink_margin: keep every sample away from the clip kinks of the surrogate and the value loss
    (log-ratio offsets either |x| < 0.05 or |x| > 0.45, value offsets |dv| < 0.05 or > 0.5, and
    |u - w| > 10 % of max(u, w)), so that the bf16 rounding of the forward pass (a few 1e-2 in
    log pi) cannot move a sample from one branch of the loss to the other; the gradient then
    differs from the FP64 one only by rounding, which is what the BF16 tolerance bounds."""
    rs = np.random.default_rng(seed)
    x, xd = _obs(M, O, Op, seed, bf16)
    p = OM.unflatten(params, O, hidden, A)
    mu, _ = OM.forward(p["actor"], x[:, :O])
    v, _ = OM.forward(p["critic"], x[:, :O])
    a = (mu + np.exp(p["log_std"]) * rs.normal(size=mu.shape)).astype(np.float32)
    off = 0.3 * rs.normal(size=M)
    dvo = 0.3 * rs.normal(size=M)
    ret = rs.normal(size=M)
    if kink_margin:
        inside = rs.random(M) < 0.5
        off = np.where(inside, rs.uniform(-0.05, 0.05, M), np.sign(rs.normal(size=M)) * rs.uniform(0.45, 0.8, M))
        inside_v = rs.random(M) < 0.5
        dvo = np.where(inside_v, rs.uniform(-0.05, 0.05, M), np.sign(rs.normal(size=M)) * rs.uniform(0.5, 1.0, M))
        vv, vo = v[:, 0], v[:, 0] - dvo
        for _ in range(50):
            vc = vo + np.clip(vv - vo, -0.2, 0.2)
            u, w_ = (vv - ret) ** 2, (vc - ret) ** 2
            bad = np.abs(u - w_) <= 0.1 * np.maximum(u, w_)
            bad &= np.abs(dvo) > 0.2
            if not bad.any():
                break
            ret[bad] = rs.normal(size=int(bad.sum())) * 2.0
    logp = OM.log_prob(a, mu, p["log_std"])
    b = {
        "obs": x, "actions": a,
        "logp_old": (logp - off).astype(np.float32),
        "mu_old": (mu + 0.05 * rs.normal(size=mu.shape)).astype(np.float32),
        "log_std_old": (p["log_std"] + 0.05).astype(np.float32),
        "v_old": (v[:, 0] - dvo).astype(np.float32),
        "adv": rs.normal(size=M).astype(np.float32), "ret": ret.astype(np.float32),
    }
    dev = {k: torch.from_numpy(np.ascontiguousarray(val)).cuda() for k, val in b.items() if k != "obs"}
    dev["obs"] = xd
    return b, dev


def _own_old_policy(L, b, d, O, params, hidden):
    """Old-policy quantities (log pi_old, V_old, mu_old) as each path produces them in training:
    the GPU side from its own inference (rl_policy_act on the same observations and parameters),
    the oracle side from its FP64 forward, with the same offsets applied to both."""
    M = b["obs"].shape[0]
    mu_g = torch.empty((M, 12), device="cuda")
    v_g = torch.empty(M, device="cuda")
    api.rl_policy_act(L.ctx, 0, d["obs"], torch.empty((M, 12), device="cuda"), mu_g, torch.empty(M, device="cuda"), v_g)
    mu_g, v_g = mu_g.cpu().numpy().astype(np.float64), v_g.cpu().numpy().astype(np.float64)
    p = OM.unflatten(params, O, hidden, 12)
    mu_o, _ = OM.forward(p["actor"], b["obs"][:, :O])
    v_o = OM.forward(p["critic"], b["obs"][:, :O])[0][:, 0]
    lp_off = OM.log_prob(b["actions"], mu_o, p["log_std"]) - b["logp_old"]     # offsets the batch chose
    dvo = v_o - b["v_old"]
    dmu = b["mu_old"] - mu_o
    gpu = dict(logp_old=(OM.log_prob(b["actions"], mu_g, p["log_std"]) - lp_off).astype(np.float32),
               v_old=(v_g - dvo).astype(np.float32), mu_old=(mu_g + dmu).astype(np.float32))
    for k, val in gpu.items():
        d[k] = torch.from_numpy(np.ascontiguousarray(val)).cuda()
    return d
