"""Pins of the scheduler oracle (MLP and features) against independent checks (no GPU).

The gradient of the MLP oracle is pinned by central finite differences of its
loss (which never calls the backpropagation code), by closed forms for
degenerate weights, and the Adam step by its first-step closed form. The
features are pinned by a hand-built two-atom pencil whose values are written
out by hand.
"""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import features, mlp


def _data(n=40, seed=3):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, mlp.N_IN))
    t = rng.standard_normal(n)
    return X, t


def test_param_count_and_layout():
    assert mlp.N_PARAM == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1 == 5313
    p = np.arange(mlp.N_PARAM, dtype=float)
    q = mlp.unpack(p)
    assert q["W1"][0, 1] == 1 and q["b1"][0] == 1024 and q["W2"][0, 0] == 1088
    assert q["b3"][0] == mlp.N_PARAM - 1


def test_gradient_matches_central_differences():
    X, t = _data()
    p = mlp.init_params(1) + 0.05 * np.random.default_rng(2).standard_normal(mlp.N_PARAM)
    g = mlp.grad(p, X, t)
    rng = np.random.default_rng(4)
    idx = np.concatenate([rng.choice(mlp.N_PARAM, 60, replace=False), [mlp.N_PARAM - 1, 0, 1024, 5248]])
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        fd = (mlp.loss(p + e, X, t) - mlp.loss(p - e, X, t)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_gradient_closed_form_zero_network():
    """All weights zero: y = b3, so dL/db3 = 2 mean(b3 - t) and every other gradient is 0."""
    X, t = _data()
    p = np.zeros(mlp.N_PARAM)
    p[-1] = 0.7
    g = mlp.grad(p, X, t)
    assert np.isclose(g[-1], 2 * np.mean(0.7 - t))
    assert np.abs(g[:-1]).max() == 0.0


def test_gradient_closed_form_constant_hidden():
    """W2 = 0: h2 = tanh(b2) for every sample, so dL/dw3 = tanh(b2) * sum_n dL/dy_n."""
    X, t = _data()
    p = mlp.init_params(5)
    q = mlp.unpack(p)
    q["W2"][...] = 0.0
    q["b2"][...] = np.linspace(-1, 1, 64)
    y, _ = mlp.forward(p, X)
    dy = 2 * (y - t) / len(t)
    g = mlp.unpack(mlp.grad(p, X, t))
    assert np.allclose(g["w3"], np.tanh(q["b2"]) * dy.sum(), rtol=1e-12, atol=1e-15)
    assert np.abs(g["W1"]).max() == 0.0     # no path from W1 to y when W2 = 0


def test_adam_first_step_is_signed_lr():
    g = np.array([0.3, -2.0, 1e-3])
    p = np.zeros(3)
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), t=1, lr=0.01)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_training_reduces_loss():
    X, t = _data(200)
    t = np.tanh(X[:, 0]) + 0.5 * X[:, 1]
    p = mlp.init_params(0)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    l0 = mlp.loss(p, X, t)
    for it in range(1, 201):
        p, m, v = mlp.adam_step(p, mlp.grad(p, X, t), m, v, it, lr=3e-3)
    assert mlp.loss(p, X, t) < 0.2 * l0


def test_features_two_atom_pencil_by_hand():
    """One C atom (rows 0-3) and one H atom (row 4) coupled only through row 4 / column 0."""
    A = np.zeros((5, 5))
    A[np.arange(4), np.arange(4)] = [-19.4, -10.7, -10.7, -10.7]
    A[4, 4] = -13.6
    A[0, 4] = A[4, 0] = -2.0
    A[1, 4] = A[4, 1] = 0.5
    B = np.eye(5)
    B[0, 4] = B[4, 0] = 0.1
    # full atom-block pattern: C block 4x4, C-H blocks, H-H
    As = sp.csr_matrix((np.array([A[i, j] for i in range(5) for j in range(5)]),
                        np.tile(np.arange(5), 5), np.arange(0, 26, 5)), shape=(5, 5))
    Bs = sp.csr_matrix((np.array([B[i, j] for i in range(5) for j in range(5)]),
                        np.tile(np.arange(5), 5), np.arange(0, 26, 5)), shape=(5, 5))
    F = features.raw_features(As, Bs, [0, 4], [4, 1], [0, 4], [0.05, 0.2])
    want0 = [np.log(0.05), 2.0, 0.05, 1 / 50, 0.0, 1 / 40, 1.0, 0.0, -1.94, 0.2, 0.1, 0.2, 19.4 ** 2 / 100,
             1.0, np.log1p(19.4 + 2.0), 1.0]
    want4 = [np.log(0.2), 0.5, 0.05, 1 / 50, 1 / 20, 0.0, 0.0, 0.0, -1.36, 0.25, 0.1,
             np.sqrt(4.25) / 10, 13.6 ** 2 / 100, 1.0, np.log1p(13.6 + 2.5), 1.0]
    assert np.allclose(F[0], want0, rtol=1e-12, atol=1e-12)
    assert np.allclose(F[1], want4, rtol=1e-12, atol=1e-12)
