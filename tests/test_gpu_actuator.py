"""The CUDA LSTM actuator cell (rl_actuator_lstm_step) against the float64 oracle
(oracle/actuator.py): four chained substeps for every joint of 4096 robots plus a ragged tail,
torques and cell state within fp32 rounding; a single joint; n = 0 leaves everything untouched."""
import numpy as np
import pytest
import torch

from oracle import actuator as OA
from paper_2109_11978_b300 import api

pytestmark = pytest.mark.gpu


def _case(n, seed):
    rng = np.random.default_rng(seed)
    w = rng.uniform(-0.3, 0.3, OA.N_WEIGHTS)
    x = rng.normal(size=(n, OA.I)) * np.array([0.3, 3.0])       # position error (rad), velocity (rad/s)
    h = rng.uniform(-0.5, 0.5, (n, OA.H))
    c = rng.normal(size=(n, OA.H))
    return w, x, h, c


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("n", [4096 * 12 + 37, 1])
def test_chained_steps_match_oracle(n):
    w, x, h, c = _case(n, 5)
    wd, hd, cd, taud = _dev(w), _dev(h), _dev(c), torch.empty(n, device="cuda")
    # the oracle starts from the same fp32-rounded values
    w, h, c = (a.astype(np.float32).astype(np.float64) for a in (w, h, c))
    for s in range(4):
        xs = x * (1.0 - 0.2 * s)
        api.rl_actuator_lstm_step(wd, _dev(xs), hd, cd, taud)
        tau, h, c = OA.step(w, xs.astype(np.float32).astype(np.float64), h, c)
        torch.cuda.synchronize()
        assert np.max(np.abs(taud.cpu().numpy() - tau)) <= 2e-5
        assert np.max(np.abs(hd.cpu().numpy() - h)) <= 2e-5
        assert np.max(np.abs(cd.cpu().numpy() - c)) <= 2e-5


def test_empty_batch_and_shapes():
    w = torch.zeros(OA.N_WEIGHTS, device="cuda")
    x, h, c, tau = (torch.ones(s, device="cuda") for s in ((0, 2), (0, 32), (0, 32), (0,)))
    api.rl_actuator_lstm_step(w, x, h, c, tau)
    torch.cuda.synchronize()
    with pytest.raises(api.RLError):
        api.rl_actuator_lstm_step(w, torch.ones((3, 3), device="cuda"), torch.ones((3, 32), device="cuda"),
                                  torch.ones((3, 32), device="cuda"), torch.ones(3, device="cuda"))
