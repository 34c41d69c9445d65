"""CPU reference of the launch-shape cost model (TEST INFRASTRUCTURE ONLY).

Plain numpy in float64, written from the model's definition: input
encoding, the two tanh layers and the linear output, the mean squared error
of log(ms) and its gradient by the chain rule.  Parameter layout (flat):
W1 (H x 16, row-major), b1 (H), W2 (H x H), b2 (H), w3 (H), b3 (1).
"""
from __future__ import annotations

import numpy as np

N_IN = 16


def encode(records) -> np.ndarray:
    x = np.zeros((len(records), N_IN))
    for i, r in enumerate(records):
        x[i, :8] = np.asarray(r.feat[:8], dtype=np.float64) / 32.0
        gemm = r.kind == 0
        x[i, 8] = 1.0 if gemm else 0.0
        x[i, 9] = 0.0 if gemm else 1.0
        if gemm and 0 <= r.param <= 2:
            x[i, 10 + r.param] = 1.0
        if not gemm:
            x[i, 13] = np.log2(max(r.param, 1)) / 4.0
        x[i, 14] = r.slot / 2.0
        x[i, 15] = float(r.precision)
    return x


def unpack(p, hidden):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + hidden * N_IN].reshape(hidden, N_IN); o += hidden * N_IN
    b1 = p[o:o + hidden]; o += hidden
    W2 = p[o:o + hidden * hidden].reshape(hidden, hidden); o += hidden * hidden
    b2 = p[o:o + hidden]; o += hidden
    w3 = p[o:o + hidden]; o += hidden
    b3 = p[o]; o += 1
    assert o == p.size
    return W1, b1, W2, b2, w3, b3


def forward(p, hidden, X):
    W1, b1, W2, b2, w3, b3 = unpack(p, hidden)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    out = h2 @ w3 + b3
    return out, (h1, h2)


def loss_and_grad(p, hidden, X, y):
    """Mean squared error of the outputs against y and its gradient."""
    W1, b1, W2, b2, w3, b3 = unpack(p, hidden)
    out, (h1, h2) = forward(p, hidden, X)
    n = X.shape[0]
    e = out - y
    loss = float(np.mean(e * e))
    d3 = 2.0 * e / n                         # dL/dout
    gw3 = h2.T @ d3
    gb3 = d3.sum()
    d2 = np.outer(d3, w3) * (1.0 - h2 * h2)  # dL/d(pre-activation 2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    gW1 = d1.T @ X
    gb1 = d1.sum(axis=0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, grad
