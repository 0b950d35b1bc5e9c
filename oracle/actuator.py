"""Batched LSTM actuator network (Sec. 3.3): one recurrent cell per joint that maps the joint's
current measurements to a torque, stepped once per simulation substep.

TEST INFRASTRUCTURE ONLY: a plain float64 numpy restatement that the CUDA kernel is checked
against; it shares no code with it and nothing on the product path imports it.

The paper states only that, following earlier actuator-network work, the torque comes from an
LSTM fed with the current measurements instead of a feed-forward net over a history of them.
Readings: the measurements are the position error q* - q and the joint velocity qd (I = 2
inputs); one LSTM layer of H = 32 units, the standard cell (Hochreiter & Schmidhuber 1997, with
a forget gate) in the gate order input, forget, cell, output:
    a = W_ih x + W_hh h + b                        (4H pre-activations)
    i = sigmoid(a_i), f = sigmoid(a_f), g = tanh(a_g), o = sigmoid(a_o)
    c' = f * c + i * g,  h' = o * tanh(c'),  tau = w_out . h' + b_out
Weights are a flat vector [W_ih (4H x I, row-major) | W_hh (4H x H) | b (4H) | w_out (H) | b_out].
The paper's trained weights are not available: the throughput runs use random ones.
"""
import numpy as np

I, H = 2, 32
N_WEIGHTS = 4 * H * I + 4 * H * H + 4 * H + H + 1


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    assert w.size == N_WEIGHTS
    o = 0
    W_ih = w[o:o + 4 * H * I].reshape(4 * H, I); o += 4 * H * I
    W_hh = w[o:o + 4 * H * H].reshape(4 * H, H); o += 4 * H * H
    b = w[o:o + 4 * H]; o += 4 * H
    w_out = w[o:o + H]; o += H
    return W_ih, W_hh, b, w_out, w[o]


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def step(w, x, h, c):
    """One cell step for n joints: x [n][I], h [n][H], c [n][H] -> (tau [n], h' [n][H], c' [n][H])."""
    W_ih, W_hh, b, w_out, b_out = unpack(w)
    x, h, c = (np.asarray(v, dtype=np.float64) for v in (x, h, c))
    a = x @ W_ih.T + h @ W_hh.T + b
    i, f, g, o = (a[:, k * H:(k + 1) * H] for k in range(4))
    c2 = sigmoid(f) * c + sigmoid(i) * np.tanh(g)
    h2 = sigmoid(o) * np.tanh(c2)
    return h2 @ w_out + b_out, h2, c2
