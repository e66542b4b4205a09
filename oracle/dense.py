"""O1 and O2: Green's-function elements from dense factorizations.

Test infrastructure only (see the package docstring).

G(z) = (z B - A)^{-1} (Sec. III-A, Eq. EQ-SHIFT-EQ and EQ-EIG-X=GB); column j
of G(z) solves (z B - A) x = e_j (Eq. EQ-SHIFT-EQ-J). Only the elements
G_ij with i in the pattern of column j of A are returned (nearsightedness,
Sec. II-B: rho_ji is needed only where X_ij != 0).

Output layout, shared with the library's contract: for the requested columns
cols[0..C), the rows of column j are the column indices of CSR row j of A in
ascending order (A is symmetric, so row j and column j have the same pattern);
the result is a flat (sum_c |P(cols[c])|, S) complex128 array, column blocks
concatenated in the order of cols.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def pattern_rows(A, j: int) -> np.ndarray:
    """Rows i of the pattern P(j): column indices of CSR row j of A."""
    return np.asarray(A.indices[A.indptr[j]:A.indptr[j + 1]], dtype=np.int64)


def pattern_offsets(A, cols) -> np.ndarray:
    cols = np.asarray(cols, dtype=np.int64)
    lens = np.diff(A.indptr)[cols]
    off = np.zeros(cols.size + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return off


def _extract(A, cols, dense_cols_per_shift) -> np.ndarray:
    """Gather G_ij, i in P(j), from dense columns G[:, c] for every shift."""
    off = pattern_offsets(A, cols)
    S = len(dense_cols_per_shift)
    out = np.empty((int(off[-1]), S), dtype=np.complex128)
    for c, j in enumerate(np.asarray(cols).tolist()):
        rows = pattern_rows(A, j)
        for k in range(S):
            out[off[c]:off[c + 1], k] = dense_cols_per_shift[k][rows, c]
    return out


def green_lu(A, B, z, cols) -> np.ndarray:
    """O1: for each shift z_k, LU-factor z_k B - A densely and solve for e_j, j in cols."""
    Ad = A.toarray()
    Bd = B.toarray()
    M = Ad.shape[0]
    cols = np.asarray(cols, dtype=np.int64)
    rhs = np.zeros((M, cols.size), dtype=np.complex128)
    rhs[cols, np.arange(cols.size)] = 1.0
    per_shift = []
    for zk in np.asarray(z, dtype=np.complex128).tolist():
        K = zk * Bd - Ad
        lu = sla.lu_factor(K, check_finite=True)
        per_shift.append(sla.lu_solve(lu, rhs))
    return _extract(A, cols, per_shift)


def generalized_eigh(A, B):
    """Eigenpairs of A y = lambda B y with y_k^T B y_l = delta_kl (Eq. EQ-GEV-EQ)."""
    lam, Y = sla.eigh(A.toarray(), B.toarray())
    return lam, Y


def green_eig(A, B, z, cols, eig=None) -> np.ndarray:
    """O2: G(z) = sum_k y_k y_k^T / (z - lambda_k) (Eq. EQ-EIG-GREEN), on the pattern."""
    lam, Y = generalized_eigh(A, B) if eig is None else eig
    cols = np.asarray(cols, dtype=np.int64)
    per_shift = []
    for zk in np.asarray(z, dtype=np.complex128).tolist():
        per_shift.append((Y / (zk - lam)[None, :]) @ Y[cols, :].T)
    return _extract(A, cols, per_shift)


def green_dense_full(A, B, zk: complex) -> np.ndarray:
    """Full dense (z B - A)^{-1} for one shift (small checks only)."""
    return np.linalg.inv(zk * B.toarray() - A.toarray())
