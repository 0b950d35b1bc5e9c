"""The allocation-free GAE entry point (rl_gae_noalloc) against rl_gae with a caller workspace.

Some callers cannot allocate device memory (a fixed memory budget reserved by another framework,
a plugin barred from the CUDA allocator, a latency-critical loop); rl_gae_noalloc serves them
with a static device scratch array.  Two calls in a row with different inputs must give the
results of the regular entry point (same kernels, so the same bits; checked against the FP32
tolerance of the other tests), with and without normalisation, and sizes past the array's limit
are refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2109_11978_b300 import api
from tests.helpers import TOL_FP32, rel_err

pytestmark = pytest.mark.gpu


def _inputs(T, N, seed):
    rs = np.random.default_rng(seed)
    cu = lambda x: torch.from_numpy(x).cuda()
    return (cu(rs.normal(size=(T, N)).astype(np.float32)), cu(rs.normal(size=(T, N)).astype(np.float32)),
            cu(rs.normal(size=N).astype(np.float32)), cu((rs.random((T, N)) < 0.05).astype(np.uint8)))


def _run(fn, T, N, args, normalize, **kw):
    adv = torch.empty((T, N), device="cuda")
    ret = torch.empty((T, N), device="cuda")
    st = torch.empty(2, device="cuda")
    fn(0.99, 0.95, *args, adv, ret, normalize=normalize, adv_stats_out=st, **kw)
    torch.cuda.synchronize()
    return adv.cpu().numpy(), ret.cpu().numpy(), st.cpu().numpy()


@pytest.mark.parametrize("T,N", [(24, 4096), (24, 1000)])
def test_noalloc_matches_regular_entry_point_twice(T, N):
    ws = torch.empty(api.rl_gae_workspace_bytes(T, N) // 4 + 4, device="cuda")
    for call, seed in enumerate((11, 12)):          # two calls in a row, different inputs
        args = _inputs(T, N, seed)
        for normalize in (True, False):
            a0, r0, s0 = _run(api.rl_gae, T, N, args, normalize, workspace=ws)
            a1, r1, s1 = _run(api.rl_gae_noalloc, T, N, args, normalize)
            assert rel_err(a1, a0) < TOL_FP32 and rel_err(r1, r0) < TOL_FP32, (call, normalize)
            assert np.allclose(s1, s0, rtol=TOL_FP32, atol=0), (call, normalize, s1, s0)


def test_noalloc_rejects_sizes_past_the_static_scratch():
    """The array holds 4096 slots: one per block of 256 robots and the (mean, std) slot, so at most
    1,048,320 robots; one more is refused, the limit itself matches the regular entry point."""
    T, NMAX = 1, 4095 * 256
    args = _inputs(T, NMAX + 1, 3)
    with pytest.raises(api.RLError):
        _run(api.rl_gae_noalloc, T, NMAX + 1, args, True)
    cut = tuple(x[..., :NMAX].contiguous() for x in args)
    a, r, s = _run(api.rl_gae_noalloc, T, NMAX, cut, True)
    ws = torch.empty(api.rl_gae_workspace_bytes(T, NMAX) // 4 + 4, device="cuda")
    a0, r0, s0 = _run(api.rl_gae, T, NMAX, cut, True, workspace=ws)
    assert np.isfinite(a).all()
    assert rel_err(a, a0) < TOL_FP32 and rel_err(r, r0) < TOL_FP32
