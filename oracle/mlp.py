"""Reference of the column scheduler's regressor: a 16 -> 64 -> 64 -> 1 MLP.

Test infrastructure only (see the package docstring).

The scheduler predicts, from per-column features, the logarithm of the number
of Lanczos steps a column needs; the queue then hands out the longest columns
first. This addresses the load imbalance from disorder that the paper
reports (Sec. IV-C: barrier time from structural disorder in the polymer runs,
with better load balance left as a future issue).

Network: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3.
Loss: mean squared error, L = (1/N) sum_n (y_n - t_n)^2.
Optimiser: Adam (Kingma and Ba, ICLR 2015) with bias correction:
m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Parameters are one flat vector in this order: W1 (64 x 16, row-major), b1 (64),
W2 (64 x 64, row-major), b2 (64), w3 (64), b3 (1).
"""

from __future__ import annotations

import numpy as np

N_IN, N_H = 16, 64
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("w3", (N_H,)), ("b3", (1,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def init_params(seed: int) -> np.ndarray:
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = np.zeros(N_PARAM)
    q = unpack(p)
    for name, (fi, fo) in (("W1", (N_IN, N_H)), ("W2", (N_H, N_H))):
        lim = np.sqrt(6.0 / (fi + fo))
        q[name][...] = rng.uniform(-lim, lim, size=q[name].shape)
    lim = np.sqrt(6.0 / (N_H + 1))
    q["w3"][...] = rng.uniform(-lim, lim, size=N_H)
    return p


def forward(p: np.ndarray, X: np.ndarray):
    q = unpack(p)
    h1 = np.tanh(X @ q["W1"].T + q["b1"])
    h2 = np.tanh(h1 @ q["W2"].T + q["b2"])
    y = h2 @ q["w3"] + q["b3"][0]
    return y, (h1, h2)


def loss(p: np.ndarray, X: np.ndarray, t: np.ndarray) -> float:
    y, _ = forward(p, X)
    return float(np.mean((y - t) ** 2))


def grad(p: np.ndarray, X: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Gradient of the mean squared error by the chain rule (backpropagation)."""
    q = unpack(p)
    y, (h1, h2) = forward(p, X)
    n = X.shape[0]
    dy = 2.0 * (y - t) / n                       # dL/dy
    g = np.zeros_like(p)
    gq = unpack(g)
    gq["w3"][...] = dy @ h2
    gq["b3"][0] = dy.sum()
    dz2 = np.outer(dy, q["w3"]) * (1.0 - h2 ** 2)     # through tanh of layer 2
    gq["W2"][...] = dz2.T @ h1
    gq["b2"][...] = dz2.sum(axis=0)
    dz1 = (dz2 @ q["W2"]) * (1.0 - h1 ** 2)
    gq["W1"][...] = dz1.T @ X
    gq["b1"][...] = dz1.sum(axis=0)
    return g


def adam_step(p, g, m, v, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
