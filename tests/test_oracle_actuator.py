"""Pins of the oracle's LSTM actuator cell: torch.nn.LSTMCell (an independent implementation of the
standard cell, same gate order) in float64, and closed forms of special weights."""
import numpy as np
import torch

from oracle import actuator as A


def _weights(rng, scale=0.3):
    return rng.uniform(-scale, scale, A.N_WEIGHTS)


def test_matches_torch_lstm_cell():
    rng = np.random.default_rng(0)
    w = _weights(rng)
    n = 257
    x, h, c = rng.normal(size=(n, A.I)), rng.normal(size=(n, A.H)), rng.normal(size=(n, A.H))
    W_ih, W_hh, b, w_out, b_out = A.unpack(w)
    cell = torch.nn.LSTMCell(A.I, A.H).double()
    with torch.no_grad():
        cell.weight_ih.copy_(torch.from_numpy(W_ih))
        cell.weight_hh.copy_(torch.from_numpy(W_hh))
        cell.bias_ih.copy_(torch.from_numpy(b))
        cell.bias_hh.zero_()
        h_t, c_t = cell(torch.from_numpy(x), (torch.from_numpy(h), torch.from_numpy(c)))
    tau, h2, c2 = A.step(w, x, h, c)
    assert np.allclose(h2, h_t.numpy(), rtol=0, atol=1e-14)
    assert np.allclose(c2, c_t.numpy(), rtol=0, atol=1e-14)
    assert np.allclose(tau, h_t.numpy() @ w_out + b_out, rtol=0, atol=1e-13)


def test_zero_weights_halve_the_cell():
    # every gate at sigmoid(0) = 1/2, g = tanh(0) = 0: c' = c / 2, h' = tanh(c / 2) / 2, tau = b_out
    w = np.zeros(A.N_WEIGHTS)
    w[-1] = 0.75
    c = np.linspace(-2, 2, 3 * A.H).reshape(3, A.H)
    tau, h2, c2 = A.step(w, np.ones((3, A.I)), np.ones((3, A.H)), c)
    assert np.array_equal(c2, c / 2)
    assert np.allclose(h2, np.tanh(c / 2) / 2, rtol=0, atol=1e-15)
    assert np.array_equal(tau, np.full(3, 0.75))


def test_saturated_gates():
    # forget gate shut and input gate open with a large cell bias: c' = tanh(big) = 1 everywhere
    w = np.zeros(A.N_WEIGHTS)
    o = 4 * A.H * A.I + 4 * A.H * A.H
    b = w[o:o + 4 * A.H]
    b[0:A.H] = 50.0           # input gate -> 1
    b[A.H:2 * A.H] = -50.0    # forget gate -> 0
    b[2 * A.H:3 * A.H] = 50.0  # cell candidate -> 1
    b[3 * A.H:] = 50.0        # output gate -> 1
    tau, h2, c2 = A.step(w, np.zeros((2, A.I)), np.zeros((2, A.H)), np.full((2, A.H), 7.0))
    assert np.allclose(c2, 1.0, atol=1e-15) and np.allclose(h2, np.tanh(1.0), atol=1e-15)
