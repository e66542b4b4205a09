"""Pins of the batched O3 oracle (oracle/krylov.py lanczos_batch, C loops in
oracle/o3_batch.c), which writes the stored references of the 100,000- and
1,000,000-atom workloads.

Tied to things other than itself:
  * the pivoted tridiagonal elimination against LAPACK's zgtsv (a library
    routine for the same system) and against a dense solve;
  * the first Lanczos steps against the one-column NumPy oracle (the same
    algorithm written independently, Sec. III-B), before finite-precision
    Lanczos iterates drift apart;
  * converged G against the definition G = (z B - A)^-1 by dense LU (O1,
    Eq. EQ-SHIFT-EQ-J) on the 64- and 1,000-atom pencils, with per-column
    damping, including the residual estimate |y_n| ||u_n||;
  * a column's result is bitwise the same alone or inside a batch, and
    with 1 or several threads (the columns share only the matrix traversal);
  * the batched sparse product and CG against SciPy's product and a dense
    solve.
"""

import numpy as np
import pytest
import scipy.linalg as la
from scipy.linalg import lapack

from oracle import dense, krylov
from paper_1609_08377_gb300 import synthetic as syn


@pytest.fixture(scope="module")
def c64():
    return syn.make_system(64, 1.0, 0)


@pytest.fixture(scope="module")
def ch1k():
    return syn.make_system(1000, 1.0 / 3.0, 0)


def test_tridiag_matches_zgtsv_and_dense():
    rng = np.random.default_rng(3)
    for n in (1, 2, 3, 7, 40):
        alpha = rng.uniform(-20, 5, n)
        beta = rng.uniform(0.5, 8, max(n - 1, 1))
        z = np.array([-3.0 + 0.05j, 1.0 + 0.2j, -19.0 + 0.1j, 4.9 + 0.07j])
        last, y = krylov.tridiag_solve_c(alpha, beta[: n - 1], 1.7, z, full=True)
        for k, zk in enumerate(z):
            T = np.diag(alpha) + np.diag(beta[: n - 1], 1) + np.diag(beta[: n - 1], -1)
            rhs = np.zeros(n, dtype=complex)
            rhs[0] = 1.7
            yd = np.linalg.solve(zk * np.eye(n) - T, rhs)
            assert np.abs(y[k] - yd).max() <= 1e-12 * np.abs(yd).max()
            assert abs(last[k] - yd[-1]) <= 1e-12 * np.abs(yd).max()
            if n > 1:
                off = (-beta[: n - 1]).astype(complex)
                _, _, _, yl, info = lapack.zgtsv(off.copy(), (zk - alpha).astype(complex), off.copy(),
                                                 rhs[:, None].copy())
                assert info == 0
                assert np.abs(y[k] - yl[:, 0]).max() <= 1e-12 * np.abs(yl).max()


def test_tridiag_pivots():
    """A zero leading pivot (z = alpha_1 exactly) forces a row interchange."""
    alpha = np.array([2.0, -1.0, 0.5])
    beta = np.array([1.0, 3.0])
    z = np.array([2.0 + 0.0j])
    last, y = krylov.tridiag_solve_c(alpha, beta, 1.0, z, full=True)
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    yd = np.linalg.solve(2.0 * np.eye(3) - T, np.array([1.0, 0, 0]))
    assert np.abs(y[0] - yd).max() <= 1e-14 * np.abs(yd).max()


def test_spmm_and_cg_against_scipy(ch1k):
    lib = krylov._o3lib()
    p = krylov._p
    A, B = ch1k.A, ch1k.B
    M, C = A.shape[0], 5
    X = np.random.default_rng(0).standard_normal((M, C))
    Y = np.zeros((M, C))
    ap, ai, av = krylov._csr_parts(A)
    lib.o3_spmm(M, p(ap), p(ai), p(av), C, C, p(X), p(Y))
    assert np.abs(Y - A @ X).max() <= 1e-12 * np.abs(A @ X).max()
    bp, bi, bv = krylov._csr_parts(B)
    V = np.zeros((M, C))
    W = [np.zeros((M, C)) for _ in range(3)]
    it = lib.o3_cg(M, p(bp), p(bi), p(bv), C, C, p(X), p(V), 1e-14, 1000, p(W[0]), p(W[1]), p(W[2]))
    assert it > 0
    Vd = la.solve(B.toarray(), X, assume_a="pos")
    assert np.abs(V - Vd).max() <= 1e-12 * np.abs(Vd).max()


def test_first_steps_match_numpy_oracle(ch1k):
    """Steps 1..12 (before rounding differences grow): alpha, beta, beta0 agree."""
    z = syn.shifts(syn.energy_grid(8), 0.1)
    cols = [0, 7, 1500]
    rb = krylov.lanczos_batch(ch1k.A, ch1k.B, cols, [z] * 3, tol=0.0, max_iter=12)
    for c, j in enumerate(cols):
        r = krylov.lanczos_column(ch1k.A, ch1k.B, j, z, tol=0.0, max_iter=12)
        assert rb[c].iters == r.iters == 12
        assert abs(rb[c].beta0 - r.beta0) <= 1e-14
        assert np.abs(rb[c].alpha - r.alpha).max() <= 1e-10
        assert np.abs(rb[c].beta - r.beta[:rb[c].beta.size]).max() <= 1e-10
        assert np.abs(rb[c].G - r.G).max() <= 1e-8 * np.abs(r.G).max()


def test_converged_matches_lu_c64(c64):
    z = syn.shifts(syn.energy_grid(16), 0.1)
    cols = np.array([0, 1, 63, 128, 200, 255])
    rb = krylov.lanczos_batch(c64.A, c64.B, cols, [z] * cols.size, tol=1e-10, max_iter=5000)
    R = dense.green_lu(c64.A, c64.B, z, cols)
    off = dense.pattern_offsets(c64.A, cols)
    for c in range(cols.size):
        assert rb[c].converged
        Rc = R[off[c]:off[c + 1]]
        assert np.abs(rb[c].G - Rc).max() <= 1e-9 * np.abs(Rc).max()


def test_converged_matches_lu_ch1k_per_column_eta(ch1k):
    eps = syn.energy_grid(16)
    cols = np.array([2, 999, 1990])
    etas = [0.2, 0.1, 0.2]
    zs = [syn.shifts(eps, e) for e in etas]
    rb = krylov.lanczos_batch(ch1k.A, ch1k.B, cols, zs, tol=1e-10, max_iter=20000, milestones=(1e-8,))
    for c, j in enumerate(cols):
        R = dense.green_lu(ch1k.A, ch1k.B, zs[c], np.array([j]))
        assert rb[c].converged and rb[c].resid.max() <= 1e-10
        assert 0 < rb[c].reached[1e-8] <= rb[c].iters
        assert np.abs(rb[c].G - R).max() <= 1e-9 * np.abs(R).max()
        # the residual estimate is the true residual of x = Q y (Eq. EQ-SHIFT-EQ-J)
    # the damping orders the step counts: larger eta converges sooner
    assert rb[0].iters < rb[1].iters and rb[2].iters < rb[1].iters


def test_alone_equals_batch_and_threads(c64):
    z = syn.shifts(syn.energy_grid(16), 0.1)
    z2 = syn.shifts(syn.energy_grid(16), 0.05)
    cols = [3, 40, 222]
    n0 = krylov.set_threads(0)
    try:
        rb = krylov.lanczos_batch(c64.A, c64.B, cols, [z, z2, z], tol=1e-10, max_iter=3000)
        krylov.set_threads(1)
        for c, j in enumerate(cols):
            ra = krylov.lanczos_batch(c64.A, c64.B, [j], [[z, z2, z][c]], tol=1e-10, max_iter=3000)[0]
            assert ra.iters == rb[c].iters
            assert np.array_equal(ra.G, rb[c].G)
    finally:
        krylov.set_threads(n0)
