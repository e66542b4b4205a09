"""Multiple Arnoldi projection for one column (Sec. III-B, Eq. EQ-LS-MULTIPLE,
EQ-EIG-GREEN-KRYLOV and EQ-PROJ-PHYS-QUANT-KRYLOV).

Test infrastructure only (see the package docstring).

For column j the pencil (A, B) is projected onto the direct sum of two Krylov
subspaces of A, one started from e_j and one from B^-1 e_j, nu/2 vectors
each. The reduced nu x nu generalized eigenproblem gives Ritz pairs
(eps_m, v_m) with v_m^T B v_n = delta_mn, and

    G^(j)(z) = sum_m v_m v_m^T / (z - eps_m)
    e_j^T rho X e_j = sum_m f(eps_m) (e_j^T v_m)(v_m^T X e_j)

so the energy integral of Eq. EQ-DM-GREEN-FN is done analytically. Both
column vectors G^(j)(z) e_j and rho^(j) e_j are reported on the pattern P(j).

This module follows those steps plainly:
  1. an orthonormal basis of each Krylov subspace by Arnoldi with Euclidean
     modified Gram-Schmidt, each new vector orthogonalised twice;
  2. B^-1 e_j by conjugate gradients on the SPD B to a 1e-15 relative
     residual (the oracle's own CG; B is well conditioned, so the solve
     is accurate to about cond(B) * 1e-15);
  3. an orthonormal basis of the sum: the second basis is projected onto the
     orthogonal complement of the first (twice), and the left singular
     vectors of the result whose singular value -- the sine of a principal
     angle between the two subspaces -- is at least RANK_TOL are appended
     (the two subspaces can share directions, e.g. when B = I);
  4. the reduced pencil (Q^T A Q, Q^T B Q) solved by scipy's generalized
     symmetric eigensolver, which returns B-normalised Ritz vectors.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as la

from .density import fermi
from .krylov import cg_solve

RANK_TOL = 1e-7      # smallest sine of a principal angle kept between the two Krylov subspaces


BREAKDOWN_TOL = 1e-13   # a Krylov sequence ends when a new direction is below this times ||A||_inf


def krylov_basis(A, b: np.ndarray, m: int) -> np.ndarray:
    """Euclidean-orthonormal basis (M x r, r <= m) of K_m(A; b) by Arnoldi;
    stops early if the subspace becomes invariant (the orthogonalised A q is
    below BREAKDOWN_TOL * ||A||_inf for a unit q)."""
    M = b.size
    Q = np.zeros((M, m))
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return Q[:, :0]
    Q[:, 0] = b / nb
    scale = float(abs(A).sum(axis=1).max())
    for k in range(1, m):
        w = A @ Q[:, k - 1]
        for _ in range(2):
            for i in range(k):
                w -= (Q[:, i] @ w) * Q[:, i]
        nw = np.linalg.norm(w)
        if nw <= BREAKDOWN_TOL * scale:
            return Q[:, :k]
        Q[:, k] = w / nw
    return Q


def principal_sines(A, B, j: int, nu: int) -> np.ndarray:
    """Sines of the principal angles between K_{nu/2}(A; B^-1 e_j) and
    K_{nu/2}(A; e_j), ascending: the quantities the rank rule compares with
    RANK_TOL."""
    M = A.shape[0]
    e = np.zeros(M)
    e[j] = 1.0
    Q1 = krylov_basis(A, e, nu // 2)
    Q2 = krylov_basis(A, cg_solve(B, e, 1e-15), nu // 2)
    for _ in range(2):
        Q2 = Q2 - Q1 @ (Q1.T @ Q2)
    return np.sort(np.linalg.svd(Q2, compute_uv=False))


def subspace_basis(A, B, j: int, nu: int, rank_tol: float = RANK_TOL, seed_tol: float = 1e-15) -> np.ndarray:
    """Orthonormal basis of K_{nu/2}(A; e_j) + K_{nu/2}(A; B^-1 e_j) (Eq. EQ-LS-MULTIPLE)."""
    if nu < 2 or nu % 2:
        raise ValueError("nu must be even and >= 2")
    M = A.shape[0]
    e = np.zeros(M)
    e[j] = 1.0
    binv_e = cg_solve(B, e, seed_tol)
    Q1 = krylov_basis(A, e, nu // 2)
    Q2 = krylov_basis(A, binv_e, nu // 2)
    for _ in range(2):
        Q2 = Q2 - Q1 @ (Q1.T @ Q2)
    if Q2.shape[1] == 0:
        return Q1
    U, s, _ = np.linalg.svd(Q2, full_matrices=False)
    return np.hstack([Q1, U[:, s >= rank_tol]])


def ritz_pairs(A, B, j: int, nu: int, rank_tol: float = RANK_TOL, seed_tol: float = 1e-15):
    """(eps, V): Ritz values (ascending) and B-orthonormal Ritz vectors (M x r).
    seed_tol is the relative CG residual of B^-1 e_j."""
    Q = subspace_basis(A, B, j, nu, rank_tol, seed_tol)
    At = Q.T @ (A @ Q)
    Bt = Q.T @ (B @ Q)
    At = (At + At.T) / 2
    Bt = (Bt + Bt.T) / 2
    eps, Y = la.eigh(At, Bt)
    return eps, Q @ Y


def marnoldi_column(A, B, j: int, nu: int, z=None, mu: float = 0.0, kT: float = 0.1,
                    rank_tol: float = RANK_TOL, seed_tol: float = 1e-15):
    """Outputs for column j on its pattern P(j) (rows of CSR row j of A, in order):

      eps    Ritz values (r,)
      rho    rho^(j)_ij = sum_m f(eps_m) (v_m)_i (v_m)_j, i in P(j)
      G      G^(j)_ij(z_k) = sum_m (v_m)_i (v_m)_j / (z_k - eps_m), shape (|P|, S) (if z given)
      w      the weights (v_m)_j (v_m)_j, so that rho_jj = sum_m f(eps_m) w_m
      q      the charges (v_m)_j (B v_m)_j, so that e_j^T rho B e_j = sum_m f(eps_m) q_m
    """
    eps, V = ritz_pairs(A, B, j, nu, rank_tol, seed_tol)
    rows = A.indices[A.indptr[j]:A.indptr[j + 1]]
    vj = V[j, :]
    f = fermi(eps, mu, kT)
    rho = V[rows, :] @ (f * vj)
    out = {"eps": eps, "rho": rho, "w": vj * vj, "q": vj * (B @ V)[j, :]}
    if z is not None:
        z = np.asarray(z, dtype=np.complex128)
        out["G"] = (V[rows, :] * vj[None, :]) @ (1.0 / (z[None, :] - eps[:, None]))
    return out
