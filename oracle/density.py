"""Density-matrix elements on the pattern from Green's-function elements.

Test infrastructure only (see the package docstring).

Fermi function (Eq. EQ-FD-FUNC): f(e) = 1 / (1 + exp((e - mu) / kT)).
Density matrix from G (Eq. EQ-DM-GREEN-FN): rho = -(1/pi) int f(e) Im G(e + i0) de.
On the shift grid z_k = e_k + i eta this integral becomes the quadrature
rho_ij = -(1/pi) sum_k w_k f(e_k) Im G_ij(z_k), with caller-given weights w_k
(trapezoid weights of the e_k grid in the workloads used here).
"""

from __future__ import annotations

import numpy as np


def fermi(e, mu: float, kT: float) -> np.ndarray:
    """f(e) evaluated with exp of a non-positive argument only (no overflow)."""
    x = (np.asarray(e, dtype=np.float64) - mu) / kT
    ex = np.exp(-np.abs(x))
    return np.where(x > 0, ex / (1.0 + ex), 1.0 / (1.0 + ex))


def density_from_green(G: np.ndarray, eps: np.ndarray, w: np.ndarray, mu: float, kT: float) -> np.ndarray:
    """rho on the pattern: G is (n_elements, S) complex, one column per shift."""
    coef = np.asarray(w, dtype=np.float64) * fermi(eps, mu, kT)
    return -(G.imag @ coef) / np.pi


def trace_with(rho: np.ndarray, X, cols, offsets) -> float:
    """Tr over the column set of rho X: sum_j sum_{i in P(j)} rho_ij X_ji (Eq. TRACE-X)."""
    total = 0.0
    for c, j in enumerate(np.asarray(cols).tolist()):
        lo, hi = X.indptr[j], X.indptr[j + 1]
        if hi - lo != offsets[c + 1] - offsets[c]:
            raise ValueError("X must share the pattern of the matrix that defines rho's layout")
        # X symmetric: X_ji = X_ij = entries of row j in the same pattern order
        total += float(rho[offsets[c]:offsets[c + 1]] @ X.data[lo:hi])
    return total
