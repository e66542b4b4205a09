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


# ---------------------------------------------------------------------------
# O3 over a batch of columns (large M): the same naive B-Lanczos as
# lanczos_column, with the sparse products, the plain CG solves and the
# pivoted tridiagonal solves in C (oracle/o3_batch.c, OpenMP). The columns of
# a batch share only the traversal of the matrix; each column's arithmetic
# is that of a one-column run, in the order of the steps above.
# ---------------------------------------------------------------------------

_O3 = None


def _o3lib():
    """Load (building on first use) the oracle's C loops."""
    global _O3
    if _O3 is None:
        import ctypes

        from . import build_c

        lib = ctypes.CDLL(build_c.build())
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.o3_set_threads.argtypes = [i32]
        lib.o3_get_threads.restype = i32
        lib.o3_spmm.argtypes = [i64, P, P, P, i32, i32, P, P]
        lib.o3_cg.argtypes = [i64, P, P, P, i32, i32, P, P, dbl, i32, P, P, P]
        lib.o3_cg.restype = i32
        lib.o3_seed.argtypes = [i64, P, P, P, i32, i32, P, dbl, i32] + [P] * 9
        lib.o3_seed.restype = i32
        lib.o3_step.argtypes = [i64, P, P, P, P, P, P, i32, i32, i32, dbl, i32] + [P] * 15
        lib.o3_step.restype = i32
        lib.o3_tridiag.argtypes = [i32, P, P, dbl, i32, P, P, P]
        _O3 = lib
    return _O3


def set_threads(n: int) -> int:
    """Threads of the C loops (0 keeps the current setting); returns the count in use."""
    lib = _o3lib()
    lib.o3_set_threads(int(n))
    return int(lib.o3_get_threads())


def _csr_parts(S):
    ptr = np.ascontiguousarray(S.indptr, dtype=np.int64)
    idx = np.ascontiguousarray(S.indices, dtype=np.int32)
    val = np.ascontiguousarray(S.data, dtype=np.float64)
    return ptr, idx, val


def _p(a: np.ndarray):
    return a.ctypes.data


def tridiag_solve_c(alpha, beta, beta0, z, full: bool = False):
    """(z_k I - T) y = beta0 e_1 for every shift z_k by the C pivoted elimination.

    Returns y_n per shift, and y (S, n) when full."""
    lib = _o3lib()
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    if b.size < max(a.size - 1, 1):
        b = np.concatenate([b, np.zeros(max(a.size - 1, 1) - b.size)])
    zz = np.ascontiguousarray(np.asarray(z, dtype=np.complex128))
    last = np.zeros(zz.size, dtype=np.complex128)
    y = np.zeros((zz.size, a.size), dtype=np.complex128) if full else None
    lib.o3_tridiag(int(a.size), _p(a), _p(b), float(beta0), int(zz.size), _p(zz), _p(last),
                   _p(y) if full else None)
    return (last, y) if full else last


def lanczos_batch(A, B, cols, z_per_col, tol: float = 1e-8, max_iter: int = 5000, check_every: int = 10,
                  bsolve_tol: float = 1e-14, milestones=(), max_cg: int = 10000, progress=None,
                  on_done=None):
    """O3 for several columns at once; returns one LanczosResult per column.

    z_per_col[c] holds the S shifts of column c (its own damping). Convergence
    is tested, as in lanczos_column, every check_every steps (and at max_iter
    or when u = 0): the residual of shift k is |y_n(z_k)| ||u_n||_2, and a
    column stops when every shift is at or below tol. Finished columns leave
    the batch, the others keep running; on_done(c, result) is called as each
    column finishes.
    """
    lib = _o3lib()
    cols = np.asarray(cols, dtype=np.int64)
    C = int(cols.size)
    M = int(A.shape[0])
    ap, ai, av = _csr_parts(A)
    bp, bi, bv = _csr_parts(B)
    ld = C
    st = {k: np.zeros((M, ld)) for k in ("q", "Bq", "Bqp", "u", "v", "R", "P", "BP")}
    beta0 = np.zeros(ld)
    beta_prev = np.zeros(ld)
    alpha = np.zeros(ld)
    beta = np.zeros(ld)
    unorm = np.zeros(ld)
    rows = [pattern_rows(A, int(j)) for j in cols]
    zc = [np.asarray(z, dtype=np.complex128) for z in z_per_col]
    active = list(range(C))
    rows_act = np.ascontiguousarray(cols[active], dtype=np.int32)
    cg = lib.o3_seed(M, _p(bp), _p(bi), _p(bv), C, ld, _p(rows_act), bsolve_tol, max_cg, _p(st["q"]),
                     _p(st["Bq"]), _p(st["Bqp"]), _p(st["u"]), _p(st["v"]), _p(st["R"]), _p(st["P"]),
                     _p(st["BP"]), _p(beta0))
    if cg < 0:
        raise RuntimeError("oracle CG did not converge on the seed")
    b0 = {c: float(beta0[t]) for t, c in enumerate(active)}
    alphas = {c: [] for c in range(C)}
    betas = {c: [] for c in range(C)}
    QP = {c: [] for c in range(C)}
    out = [None] * C
    reached = {c: {} for c in range(C)}
    n = 0
    while active:
        n += 1
        na = len(active)
        off = np.zeros(na + 1, dtype=np.int64)
        for t, c in enumerate(active):
            off[t + 1] = off[t] + rows[c].size
        prow = np.ascontiguousarray(np.concatenate([rows[c] for c in active]), dtype=np.int32)
        qp = np.zeros(int(off[-1]))
        cg = lib.o3_step(M, _p(ap), _p(ai), _p(av), _p(bp), _p(bi), _p(bv), na, ld, int(n == 1), bsolve_tol,
                         max_cg, _p(st["q"]), _p(st["Bq"]), _p(st["Bqp"]), _p(st["u"]), _p(st["v"]),
                         _p(st["R"]), _p(st["P"]), _p(st["BP"]), _p(beta_prev), _p(alpha), _p(beta),
                         _p(unorm), _p(off), _p(prow), _p(qp))
        if cg < 0:
            raise RuntimeError(f"oracle CG did not converge at step {n}")
        finished = []
        for t, c in enumerate(active):
            if n > 1:
                betas[c].append(float(beta[t]))
            alphas[c].append(float(alpha[t]))
            QP[c].append(qp[off[t]:off[t + 1]].copy())
            un = float(unorm[t])
            if not (n % check_every == 0 or n == max_iter or un == 0.0):
                continue
            last = tridiag_solve_c(alphas[c], betas[c], b0[c], zc[c])
            resid = np.abs(last) * un
            for m in milestones:
                if m not in reached[c] and resid.max() <= m:
                    reached[c][m] = n
            conv = bool(np.all(resid <= tol)) or un == 0.0
            if conv or n == max_iter:
                _, y = tridiag_solve_c(alphas[c], betas[c], b0[c], zc[c], full=True)
                G = np.stack(QP[c], axis=1) @ y.T
                r = LanczosResult(G, n, resid, conv, np.asarray(alphas[c]), np.asarray(betas[c]), b0[c])
                r.reached = reached[c]
                out[c] = r
                QP[c] = None
                if on_done is not None:
                    on_done(c, r)
                finished.append(t)
        if finished:
            keep = [t for t in range(na) if t not in finished]
            for k in st:
                st[k][:, :len(keep)] = st[k][:, keep]
            for arr in (beta_prev,):
                arr[:len(keep)] = arr[keep]
            active = [active[t] for t in keep]
        if progress is not None:
            progress(n, len(active))
    return out
