"""O3 and O3': Krylov-subspace oracles for large M (column subsets).

Test infrastructure only (see the package docstring).

O3 -- naive FP64 shifted Lanczos in the B inner product (Sec. III-B: one
Krylov subspace serves every shift z_k of the generalized shifted equations
(z_k B - A) x = e_j, Eq. EQ-SHIFT-EQ-J). Written from the mathematics, not
from any listing:

  The pencil is turned into the operator H = B^{-1} A, which is self-adjoint
  in the inner product <x, y>_B = x^T B y; (z B - A) x = e_j is equivalent to
  (z I - H) x = B^{-1} e_j. Lanczos on H from b = B^{-1} e_j gives
  B-orthonormal q_1..q_n and a real tridiagonal T_n (alpha on the diagonal,
  beta off it) with A Q_n = B Q_n T_n + beta_n B q_{n+1} e_n^T.
  Then x_n(z) = Q_n y(z), (z I - T_n) y(z) = beta_0 e_1, beta_0 = ||b||_B, and
  the residual is e_j - (z B - A) x_n = y_n(z) * beta_n B q_{n+1}, whose
  2-norm is |y_n(z)| * ||u_n||_2 with u_n = beta_n B q_{n+1}.

  The oracle keeps B q alongside q, so every step needs one product with A and
  one solve with B (plain CG), and solves each shift's tridiagonal system with
  LAPACK's pivoted zgtsv -- a different route from a recurrence on an LDL^T
  factorisation.

O3' -- plain COCG on the complex-symmetric z B - A, one shift at a time, with
no B^{-1} and no shared subspace: an independent spot check of single (j, k).
"""

from __future__ import annotations

import numpy as np
from scipy.linalg import lapack

from .dense import pattern_rows


def cg_solve(B, U: np.ndarray, tol: float = 1e-14, max_iter: int = 10000) -> np.ndarray:
    """Plain conjugate gradients for B V = U, column by column (masked).

    Stops a column when ||U - B V||_2 <= tol * ||U||_2.
    """
    U = np.asarray(U, dtype=np.float64)
    one = U.ndim == 1
    if one:
        U = U[:, None]
    V = np.zeros_like(U)
    R = U.copy()
    P = R.copy()
    rr = np.einsum("ij,ij->j", R, R)
    target = (tol ** 2) * np.einsum("ij,ij->j", U, U)
    active = rr > target
    for _ in range(max_iter):
        if not active.any():
            break
        a_idx = np.nonzero(active)[0]
        Pa = P[:, a_idx]
        BP = B @ Pa
        pBp = np.einsum("ij,ij->j", Pa, BP)
        a = rr[a_idx] / pBp
        V[:, a_idx] += Pa * a
        R[:, a_idx] -= BP * a
        rr_new = np.einsum("ij,ij->j", R[:, a_idx], R[:, a_idx])
        b = rr_new / rr[a_idx]
        P[:, a_idx] = R[:, a_idx] + P[:, a_idx] * b
        rr[a_idx] = rr_new
        active[a_idx] = rr_new > target[a_idx]
    return V[:, 0] if one else V


def _tridiag_solve(alpha, beta, beta0, z):
    """Solve (z I - T) y = beta0 e_1 for one shift with LAPACK zgtsv (pivoted)."""
    n = alpha.size
    if n == 1:
        return np.array([beta0 / (z - alpha[0])], dtype=np.complex128)
    d = (z - alpha).astype(np.complex128)
    off = (-beta[: n - 1]).astype(np.complex128)
    rhs = np.zeros((n, 1), dtype=np.complex128)
    rhs[0, 0] = beta0
    _, _, _, y, info = lapack.zgtsv(off.copy(), d, off.copy(), rhs)
    if info != 0:
        raise np.linalg.LinAlgError(f"zgtsv failed, info={info}")
    return y[:, 0]


class LanczosResult:
    def __init__(self, G, iters, resid, converged, alpha, beta, beta0, x_full=None):
        self.G = G                  # (|P(j)|, S) complex128
        self.iters = iters          # Lanczos steps taken
        self.resid = resid          # (S,) residual estimate |y_n| * ||u_n||
        self.converged = converged
        self.alpha = alpha
        self.beta = beta
        self.beta0 = beta0
        self.x_full = x_full        # (M, S) when requested


def lanczos_column(A, B, j: int, z, tol: float = 1e-8, max_iter: int = 5000,
                   check_every: int = 10, bsolve_tol: float = 1e-14,
                   keep_full: bool = False, milestones=()) -> LanczosResult:
    """O3 for one column j and all shifts z (eta may differ per shift).

    milestones: residual levels above tol; the result's `reached` maps each to
    the first checked step whose largest residual estimate was at or below it.
    """
    z = np.asarray(z, dtype=np.complex128)
    M = A.shape[0]
    rows = pattern_rows(A, j)
    u = np.zeros(M)
    u[j] = 1.0
    v = cg_solve(B, u, tol=bsolve_tol)
    beta0 = float(np.sqrt(u @ v))
    q = v / beta0
    Bq = u / beta0
    Bq_prev = np.zeros(M)
    beta_prev = 0.0
    alphas, betas, QP, Qfull = [], [], [], []
    y_all = None
    resid = np.full(z.size, np.inf)
    n = 0
    converged = False
    reached = {}
    while n < max_iter:
        n += 1
        w = A @ q
        alpha = float(q @ w)
        u = w - alpha * Bq - beta_prev * Bq_prev
        alphas.append(alpha)
        QP.append(q[rows].copy())
        if keep_full:
            Qfull.append(q.copy())
        unorm = float(np.linalg.norm(u))
        if n % check_every == 0 or n == max_iter or unorm == 0.0:
            a = np.asarray(alphas)
            b = np.asarray(betas)
            y_all = np.stack([_tridiag_solve(a, b, beta0, zk) for zk in z], axis=1)
            resid = np.abs(y_all[-1, :]) * unorm
            for m in milestones:
                if m not in reached and resid.max() <= m:
                    reached[m] = n
            if np.all(resid <= tol):
                converged = True
                break
        if unorm == 0.0:        # invariant subspace: the residual is exactly 0
            converged = True
            break
        v = cg_solve(B, u, tol=bsolve_tol)
        beta = float(np.sqrt(u @ v))
        betas.append(beta)
        Bq_prev, Bq = Bq, u / beta
        q = v / beta
        beta_prev = beta
    QPm = np.stack(QP, axis=1)                 # (|P|, n)
    G = QPm @ y_all
    x_full = None
    if keep_full:
        x_full = np.stack(Qfull, axis=1) @ y_all
    res = LanczosResult(G, n, resid, converged, np.asarray(alphas), np.asarray(betas), beta0, x_full)
    res.reached = reached
    return res


def lanczos_columns(A, B, cols, z_per_col, tol=1e-8, max_iter=5000, check_every=10,
                    bsolve_tol=1e-14):
    """O3 over a list of columns; z_per_col[c] holds the S shifts of column c."""
    Gs, iters, res, conv = [], [], [], []
    for c, j in enumerate(np.asarray(cols).tolist()):
        r = lanczos_column(A, B, j, z_per_col[c], tol=tol, max_iter=max_iter,
                           check_every=check_every, bsolve_tol=bsolve_tol)
        Gs.append(r.G)
        iters.append(r.iters)
        res.append(r.resid)
        conv.append(r.converged)
    return np.concatenate(Gs, axis=0), np.asarray(iters), res, np.asarray(conv)


def cocg_solve(A, B, j: int, zk: complex, tol: float = 1e-12, max_iter: int = 100000):
    """O3': conjugate orthogonal CG on K = z B - A (complex symmetric), b = e_j.

    Uses the unconjugated bilinear form r^T r; stops at ||r||_2 <= tol.
    Returns the full solution x and the iteration count.
    """
    M = A.shape[0]
    K = (zk * B - A).tocsr()
    x = np.zeros(M, dtype=np.complex128)
    r = np.zeros(M, dtype=np.complex128)
    r[j] = 1.0
    p = r.copy()
    rho = r @ r
    for it in range(1, max_iter + 1):
        Kp = K @ p
        mu = p @ Kp
        a = rho / mu
        x += a * p
        r -= a * Kp
        if np.linalg.norm(r) <= tol:
            return x, it
        rho_new = r @ r
        p = r + (rho_new / rho) * p
        rho = rho_new
    return x, max_iter
