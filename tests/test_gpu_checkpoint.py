"""Checkpoint and resume of the whole learner (rl_checkpoint_*): a run resumed from an image
continues bit for bit, so after more iterations its parameters, env state, scalars, curriculum
levels and per-iteration statistics equal those of the saved run that kept going; images of
another config, with a damaged header or cut short are refused and leave the context as it was."""
import pytest
import torch

from paper_2109_11978_b300 import api, synth
from tests.helpers import lib_config, obs_dims, workload

pytestmark = pytest.mark.gpu


def _learner(w, tiles=None):
    cfg = lib_config(w)
    O, _ = obs_dims(w)
    params = synth.xavier_params(w["seed"] + 1, O, w["hidden"], 12, log_std=-0.3, bias_scale=0.1)
    hf = synth.heightfield(w["seed"] + 2) if w["grid"][0] else None
    L = api.Learner(cfg, hf, params)
    for t in tiles or ():
        api.rl_set_gemm_tiles(L.ctx, *t)
    return L


def _snapshot(L):
    torch.cuda.synchronize()
    sf, si = L.get_state()
    return {"params": L.params().cpu(), "sf": sf.cpu(), "si": si.cpu(), "levels": L.storage(11).clone().cpu(),
            "obs0": L.storage(0)[0].float().cpu(), "scalars": api.rl_get_scalars(L.ctx)}


def _run(L, n):
    stats = []
    for _ in range(n):
        s = torch.zeros(api.RL_NSTATS, dtype=torch.float32).pin_memory()
        api.rl_train_iteration(L.ctx, True, s)
        torch.cuda.synchronize()
        stats.append(s.clone())
    return stats


def _equal(a, b):
    for k in a:
        if k == "scalars":
            assert a[k] == b[k], k
        else:
            assert torch.equal(a[k], b[k]), k


# the second case pins split-K counts away from the defaults: the image carries them, and the
# resumed context (created with the defaults) must take them over to repeat the sums' order
@pytest.mark.parametrize("precision,tiles", [(0, None), (1, None), (1, [(2, 0, 64, 1, 5), (2, 1, 64, 1, 2)])])
def test_resume_is_bit_exact(precision, tiles):
    w = workload("small_rough", precision=precision, epochs=2, minibatches=2)
    A = _learner(w, tiles)
    _run(A, 2)
    image = api.rl_checkpoint_save(A.ctx)
    assert image.numel() == api.rl_checkpoint_bytes(A.ctx)
    stats_a = _run(A, 3)
    snap_a = _snapshot(A)
    B = _learner(w)                      # fresh context, default tile shapes, initial weights
    api.rl_checkpoint_load(B.ctx, image)
    stats_b = _run(B, 3)
    snap_b = _snapshot(B)
    _equal(snap_a, snap_b)
    # the statistics of the update are reduced in a fixed order and match exactly; the mean reward
    # (index 7) sums per-block partials with float atomics, whose order varies from run to run
    for x, y in zip(stats_a, stats_b):
        keep = torch.ones_like(x, dtype=torch.bool)
        keep[7] = False
        assert torch.equal(x[keep], y[keep])
        assert abs(float(x[7]) - float(y[7])) <= 1e-6 * max(1.0, abs(float(x[7])))
    assert snap_a["scalars"]["iteration"] == 5
    assert api.rl_last_device_status(A.ctx) == 0 and api.rl_last_device_status(B.ctx) == 0
    A.close()
    B.close()


def test_refuses_foreign_or_damaged_images():
    w = workload("small_rough", precision=1)
    A = _learner(w)
    _run(A, 1)
    image = api.rl_checkpoint_save(A.ctx)
    B = _learner(w)
    before = _snapshot(B)
    bad_magic = image.clone()
    bad_magic[0] ^= 0xFF
    bad_version = image.clone()
    bad_version[8] ^= 0x01
    for bad in (bad_magic, bad_version, image[: image.numel() - 1].clone(), image[:16].clone()):
        with pytest.raises(api.RLError):
            api.rl_checkpoint_load(B.ctx, bad)
    other = _learner(workload("small_rough", precision=1, seed=7))     # another seed: another config
    with pytest.raises(api.RLError):
        api.rl_checkpoint_load(other.ctx, image)
    with pytest.raises(api.RLError):
        api.rl_checkpoint_load(B.ctx, image.cuda())
    _equal(before, _snapshot(B))
    for L in (A, B, other):
        L.close()


def test_damaged_tile_record_leaves_the_context_as_it_was():
    """The image's GEMM tile records are all checked before any is applied: an image whose first
    record asks for another valid shape and whose last record is invalid is refused, and the
    context keeps its own shapes (its image is unchanged byte for byte)."""
    w = workload("small_rough", precision=1)
    A = _learner(w)
    _run(A, 1)
    image = api.rl_checkpoint_save(A.ctx)
    B = _learner(w)
    before = api.rl_checkpoint_save(B.ctx)
    tiles = 8 + 4 + 4 + 9 * 8                   # magic, version, segment count, segment sizes
    rec = lambda layer, site, k: tiles + ((layer * 4 + site) * 3 + k) * 4
    bad = image.clone()
    first = bad[rec(0, 0, 0):rec(0, 0, 0) + 4].view(torch.int32)
    assert int(first[0]) in (64, 128)
    first[0] = 64 if int(first[0]) == 128 else 128               # another valid width of layer 0's forward
    last = bad[rec(1, 3, 1):rec(1, 3, 1) + 4].view(torch.int32)
    last[0] = 2                                                   # cluster mode 2 is not offered
    with pytest.raises(api.RLError):
        api.rl_checkpoint_load(B.ctx, bad)
    assert torch.equal(api.rl_checkpoint_save(B.ctx), before)
    A.close()
    B.close()


def test_env_state_through_host_buffers_is_exact():
    """The env-state calls take pinned host buffers as well as device ones: the state read into
    host memory equals the one read on the device, and a training run whose state makes the round
    trip through host memory every iteration (in before, out after) repeats the device-resident
    run bit for bit (parameters, env state, the update's statistics; the mean reward sums
    per-block partials with float atomics and matches to rounding)."""
    w = workload("small_rough", precision=1)
    La, Lb = _learner(w), _learner(w)
    N = w["num_envs"]
    sf_h = torch.empty((api.RL_NF, N), dtype=torch.float32).pin_memory()
    si_h = torch.empty((api.RL_NI, N), dtype=torch.int32).pin_memory()
    api.rl_env_get_state(Lb.ctx, sf_h, si_h)
    torch.cuda.synchronize()
    sf_d, si_d = Lb.get_state()
    assert torch.equal(sf_h, sf_d.cpu()) and torch.equal(si_h, si_d.cpu())
    ref = _run(La, 2)
    got = []
    for _ in range(2):
        api.rl_env_set_state(Lb.ctx, sf_h, si_h)
        s = torch.zeros(api.RL_NSTATS, dtype=torch.float32).pin_memory()
        api.rl_train_iteration(Lb.ctx, True, s)
        api.rl_env_get_state(Lb.ctx, sf_h, si_h)
        torch.cuda.synchronize()
        got.append(s.clone())
    a, b = _snapshot(La), _snapshot(Lb)
    assert torch.equal(a["params"], b["params"])
    assert torch.equal(a["sf"], sf_h) and torch.equal(a["si"], si_h)
    for x, y in zip(ref, got):
        keep = torch.ones_like(x, dtype=torch.bool)
        keep[7] = False
        assert torch.equal(x[keep], y[keep])
        assert abs(float(x[7]) - float(y[7])) <= 1e-6 * max(1.0, abs(float(x[7])))
    assert api.rl_last_device_status(Lb.ctx) == 0
    La.close()
    Lb.close()
