"""The failure path of the bounded device waits, exercised without faulting, trapping or hanging the
GPU: a wait on an mbarrier that nothing arrives on runs out after its 2 s bound, RL_ERR_TIMEOUT
reaches the context's status word, and after the word is cleared the context computes exactly as
before (policy inference bit for bit, a training iteration with a clean status)."""
import time

import pytest
import torch

from paper_2109_11978_b300 import _native as N
from paper_2109_11978_b300 import api
from tests.gpu_helpers import _obs, _setup
from tests.helpers import workload

pytestmark = pytest.mark.gpu


def _act(L, xd, rows):
    out = [torch.empty((rows, 12), device="cuda"), torch.empty((rows, 12), device="cuda"),
           torch.empty(rows, device="cuda"), torch.empty(rows, device="cuda")]
    api.rl_policy_act(L.ctx, 2, xd, *out)
    torch.cuda.synchronize()
    return out


def test_forced_timeout_reaches_the_status_word_and_the_context_recovers():
    w = workload("tiny", precision=1)
    L, _, O, Op = _setup(w)
    _, xd = _obs(64, O, Op, 9, True)
    before = _act(L, xd, 64)
    assert api.rl_last_device_status(L.ctx) == 0
    t0 = time.time()
    api.rl_diag_forced_timeout(L.ctx)
    assert api.rl_last_device_status(L.ctx) == N.RL_ERR_TIMEOUT
    waited = time.time() - t0
    assert 1.5 < waited < 60.0, waited
    # the first failure recorded wins until the word is cleared
    api.rl_diag_forced_timeout(L.ctx)
    assert api.rl_last_device_status(L.ctx) == N.RL_ERR_TIMEOUT
    api.rl_clear_device_status(L.ctx)
    assert api.rl_last_device_status(L.ctx) == 0
    after = _act(L, xd, 64)
    for a, b in zip(before, after):
        assert torch.equal(a, b)
    L.train_iteration(use_graph=True)
    torch.cuda.synchronize()
    assert api.rl_last_device_status(L.ctx) == 0
    L.close()
