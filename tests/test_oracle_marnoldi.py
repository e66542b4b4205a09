"""Pins of the multiple Arnoldi oracle (Sec. III-B) against facts the
mathematics fixes: exactness when the subspace is the whole space, the
conservation laws that the B^-1 e_j half of the subspace enforces, the
Rayleigh-Ritz bounds and nesting, closed forms for invariant subspaces, the
Galerkin definition of G^(j), and the analytic energy integral against a
quadrature of G^(j)."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dense, density, marnoldi as ma
from paper_1609_08377_gb300 import synthetic as syn


@pytest.fixture(scope="module")
def c64():
    return syn.make_system(64, 1.0, 0)


def _pencil(M, seed):
    rng = np.random.default_rng(seed)
    A = rng.uniform(-3, 3, (M, M))
    A = (A + A.T) / 2
    E = rng.uniform(-1, 1, (M, M))
    E = (E + E.T) / 2
    np.fill_diagonal(E, 0)
    E *= 0.6 / np.abs(E).sum(axis=1).max()
    return sp.csr_matrix(A), sp.csr_matrix(np.eye(M) + E)


def test_full_space_is_exact():
    """nu/2 = M: K(A; e_j) is the whole space, so G^(j) and rho^(j) are the
    exact column (Eq. EQ-PROJ-PHYS-QUANT-KRYLOV becomes exact at nu = M)."""
    M = 10
    A, B = _pencil(M, 4)
    lam, Y = dense.generalized_eigh(A, B)
    z = np.array([-1.0 + 0.3j, 0.5 + 0.05j, 2.0 + 1.0j])
    mu, kT = 0.2, 0.3
    for j in (0, 3, 9):
        o = ma.marnoldi_column(A, B, j, 2 * M, z=z, mu=mu, kT=kT)
        assert np.allclose(o["eps"], lam, atol=1e-11)
        rho = Y @ (density.fermi(lam, mu, kT) * Y[j, :])
        Gx = dense.green_eig(A, B, z, [j])
        assert np.abs(o["rho"] - rho).max() < 1e-11
        assert np.abs(o["G"] - Gx).max() < 1e-10 * np.abs(Gx).max()


@pytest.mark.parametrize("j", [0, 17, 130, 255])
def test_conservation_laws(c64, j):
    """With e_j and B^-1 e_j in the subspace, for any nu (f = 1):
      sum_m v_m (v_m)_j        = B^-1 e_j          (every row)
      sum_m (v_m)_j (B v_m)_j  = 1
      sum_m eps_m (v_m)_j^2    = (B^-1 A B^-1)_jj
      sum_m eps_m (v_m)_j (B v_m)_j = (B^-1 A)_jj"""
    A, B = c64.A, c64.B
    # the laws are exact for the full sum of the two subspaces: keep every
    # numerically independent direction here
    eps, V = ma.ritz_pairs(A, B, j, 30, rank_tol=1e-13)
    Bd, Ad = B.toarray(), A.toarray()
    Binv = np.linalg.inv(Bd)
    vj = V[j, :]
    BV = Bd @ V
    assert np.abs(V @ vj - Binv[:, j]).max() < 1e-12
    assert abs(vj @ BV[j, :] - 1.0) < 1e-12
    assert abs((eps * vj) @ vj - (Binv @ Ad @ Binv)[j, j]) < 1e-11
    assert abs((eps * vj) @ BV[j, :] - (Binv @ Ad)[j, j]) < 1e-11
    # B-orthonormal Ritz vectors that diagonalise A on the subspace
    assert np.abs(V.T @ BV - np.eye(V.shape[1])).max() < 1e-12
    assert np.abs(V.T @ (Ad @ V) - np.diag(eps)).max() < 1e-10
    # with the default rank rule directions within sin(theta) < 1e-7 of the
    # first subspace are dropped: the laws then hold to about that size
    o = ma.marnoldi_column(A, B, j, 30)
    assert abs(o["q"].sum() - 1.0) < 1e-6


def test_ritz_bounds_and_nesting(c64):
    """Ritz values lie in [lambda_min, lambda_max]; the subspaces are nested
    in nu, so the lowest Ritz value can only fall and the highest only rise."""
    A, B = c64.A, c64.B
    lam, _ = dense.generalized_eigh(A, B)
    lo, hi = [], []
    for nu in (4, 10, 20, 30, 40):
        eps, _ = ma.ritz_pairs(A, B, 5, nu)
        assert eps.min() >= lam.min() - 1e-10 and eps.max() <= lam.max() + 1e-10
        lo.append(eps.min())
        hi.append(eps.max())
    assert all(b <= a + 1e-12 for a, b in zip(lo, lo[1:]))
    assert all(b >= a - 1e-12 for a, b in zip(hi, hi[1:]))


def test_isolated_orbital_closed_form():
    """A row with no off-diagonal entries: the subspace is span(e_j) (rank 1),
    eps = A_jj / B_jj, rho_jj = f(eps) / B_jj."""
    M = 6
    A, B = _pencil(M, 1)
    A, B = A.toarray(), B.toarray()
    A[2, :] = A[:, 2] = 0.0
    B[2, :] = B[:, 2] = 0.0
    A[2, 2], B[2, 2] = -4.0, 1.7
    A, B = sp.csr_matrix(A), sp.csr_matrix(B)
    o = ma.marnoldi_column(A, B, 2, 8, mu=-1.0, kT=0.4)
    assert o["eps"].size == 1
    assert np.isclose(o["eps"][0], -4.0 / 1.7, rtol=1e-14)
    rows = A.indices[A.indptr[2]:A.indptr[3]]
    assert list(rows) == [2]
    assert np.isclose(o["rho"][0], density.fermi(-4.0 / 1.7, -1.0, 0.4) / 1.7, rtol=1e-13)


def test_identity_overlap_has_half_rank(c64):
    """B = I: B^-1 e_j = e_j, the two Krylov subspaces coincide and the rank
    is nu/2; the conservation law sum_m v_m (v_m)_j = e_j still holds."""
    A = c64.A
    I = sp.identity(c64.M, format="csr")
    eps, V = ma.ritz_pairs(A, I, 9, 20)
    assert V.shape[1] == 10
    e = np.zeros(c64.M)
    e[9] = 1.0
    assert np.abs(V @ V[9, :] - e).max() < 1e-12


def test_green_is_the_galerkin_solution(c64):
    """G^(j)(z) e_j equals the Galerkin solution Q (Q^T (zB - A) Q)^-1 Q^T e_j
    on any basis Q of the subspace; here Q comes from the monomial vectors
    A^k e_j, A^k B^-1 e_j (k < 3) through a QR factorisation."""
    A, B = c64.A, c64.B
    j, nu = 40, 6
    z = syn.shifts(np.array([-20.0, -11.0, -3.0, 2.0]), 0.1)
    o = ma.marnoldi_column(A, B, j, nu, z=z)
    e = np.zeros(c64.M)
    e[j] = 1.0
    b2 = np.linalg.solve(B.toarray(), e)
    K = np.column_stack([e, A @ e, A @ (A @ e), b2, A @ b2, A @ (A @ b2)])
    Q, _ = np.linalg.qr(K)
    rows = A.indices[A.indptr[j]:A.indptr[j + 1]]
    for k, zk in enumerate(z):
        Mk = Q.T @ ((zk * B - A) @ Q)
        x = Q @ np.linalg.solve(Mk, Q.T @ e)
        assert np.abs(o["G"][:, k] - x[rows]).max() < 1e-11 * np.abs(x).max()


def test_analytic_integral_matches_quadrature(c64):
    """-(1/pi) Im G^(j)(e + i eta) is a sum of Lorentzians of width eta at the
    Ritz values with weights c_m = (v_m)_i (v_m)_j (Eq. EQ-EIG-GREEN-KRYLOV), so
    the quadrature of f against it on a fine grid equals sum_m c_m F(eps_m),
    F = f smoothed by the Lorentzian (computed here by adaptive integration).
    As eta -> 0, F -> f, which is the analytic sum of
    Eq. EQ-PROJ-PHYS-QUANT-KRYLOV."""
    from scipy import integrate

    A, B = c64.A, c64.B
    j, nu, mu, kT, eta = 11, 30, -10.0, 0.2, 0.01
    eps_r, V = ma.ritz_pairs(A, B, j, nu)
    lo, hi = eps_r.min() - 20, eps_r.max() + 20
    grid = np.linspace(lo, hi, int(np.ceil((hi - lo) / (eta / 8))) + 1)
    w = syn.trapezoid_weights(grid)
    z = syn.shifts(grid, eta)
    o = ma.marnoldi_column(A, B, j, nu, z=z, mu=mu, kT=kT)
    quad = density.density_from_green(o["G"], grid, w, mu, kT)
    rows = A.indices[A.indptr[j]:A.indptr[j + 1]]
    c = V[rows, :] * V[j, :][None, :]

    def smoothed(e0):
        fn = lambda e: density.fermi(e, mu, kT) * (eta / np.pi) / ((e - e0) ** 2 + eta ** 2)
        pts = sorted({float(e0), float(mu)})
        val, _ = integrate.quad(fn, lo, hi, points=pts, limit=2000, epsabs=1e-13, epsrel=1e-12)
        return val

    F = np.array([smoothed(e) for e in eps_r])
    assert np.abs(quad - c @ F).max() < 1e-8
    f = density.fermi(eps_r, mu, kT)
    assert np.all(np.abs(quad - o["rho"]) <= np.abs(c) @ np.abs(F - f) + 1e-8)
    assert np.abs(F - f).max() < 0.05       # the smoothing is a small correction at eta = 0.01


@pytest.mark.parametrize("mu,kT", [(-10.0, 0.1), (-2.0, 0.5), (5.0, 0.05)])
def test_rho_trace_equals_weighted_charges(c64, mu, kT):
    """e_j^T rho^(j) B e_j two ways (Eq. EQ-PROJ-PHYS-QUANT-KRYLOV with X = B):
    through rho on the pattern, sum_i rho_ij B_ij, and through the Ritz
    charges, sum_m f(eps_m) (v_m)_j (B v_m)_j; and with X = A the energy
    sum_i rho_ij A_ij equals sum_m f(eps_m) eps_m (v_m)_j (B v_m)_j."""
    A, B = c64.A, c64.B
    for j in (2, 64, 200):
        o = ma.marnoldi_column(A, B, j, 30, mu=mu, kT=kT)
        lo, hi = A.indptr[j], A.indptr[j + 1]
        f = density.fermi(o["eps"], mu, kT)
        via_rho_B = float(o["rho"] @ B.data[lo:hi])
        via_rho_A = float(o["rho"] @ A.data[lo:hi])
        assert abs(via_rho_B - f @ o["q"]) <= 1e-12 * max(1.0, abs(via_rho_B))
        assert abs(via_rho_A - (f * o["eps"]) @ o["q"]) <= 1e-11 * max(1.0, abs(via_rho_A))
