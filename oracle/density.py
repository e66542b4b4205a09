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


# ---------------------------------------------------------------------------
# Trace quantities on the shift grid and the chemical potential
# ---------------------------------------------------------------------------

def shift_traces(G: np.ndarray, X, cols, offsets) -> np.ndarray:
    """s_k = sum_j sum_{i in P(j)} Im G_ij(z_k) X_ji, one number per shift.

    With these, Tr(rho X) = -(1/pi) sum_k w_k f(e_k) s_k for any mu, so the
    electron count (X = B) as a function of mu costs O(S) per evaluation.
    """
    S = G.shape[1]
    s = np.zeros(S)
    for c, j in enumerate(np.asarray(cols).tolist()):
        lo, hi = X.indptr[j], X.indptr[j + 1]
        if hi - lo != offsets[c + 1] - offsets[c]:
            raise ValueError("X must share the pattern of the matrix that defines G's layout")
        s += X.data[lo:hi] @ G[offsets[c]:offsets[c + 1]].imag
    return s


def count_from_traces(s: np.ndarray, eps: np.ndarray, w: np.ndarray, mu: float, kT: float) -> float:
    """N(mu) = -(1/pi) sum_k w_k f(e_k) s_k (Eq. TRACE-X with X = B, by quadrature)."""
    return float(-(np.asarray(w) * fermi(eps, mu, kT)) @ s / np.pi)


def find_mu(s, eps, w, kT: float, n_elec: float, lo: float, hi: float, iters: int = 200) -> float:
    """mu with N(mu) = n_elec by plain bisection on [lo, hi] (Sec. II: mu is fixed
    by the number of electrons). Requires N(lo) < n_elec <= N(hi); keeps that
    invariant, so it returns a root of the continuous N in the bracket."""
    nlo = count_from_traces(s, eps, w, lo, kT)
    nhi = count_from_traces(s, eps, w, hi, kT)
    if not (nlo < n_elec <= nhi):
        raise ValueError(f"n_elec={n_elec} not bracketed: N(lo)={nlo}, N(hi)={nhi}")
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if count_from_traces(s, eps, w, mid, kT) >= n_elec:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def atom_pattern(A, orb_offset, orb_count):
    """Atom-pair pattern of A: for atom J, the sorted atoms I with some A_{Ia,Jb}
    in the pattern. Returns (aptr, aidx) in CSR form over atoms."""
    n_atoms = len(orb_offset)
    atom_of = np.repeat(np.arange(n_atoms), np.asarray(orb_count, dtype=np.int64))
    aptr = [0]
    aidx = []
    for J in range(n_atoms):
        nb = set()
        for b in range(int(orb_count[J])):
            j = int(orb_offset[J]) + b
            nb.update(atom_of[A.indices[A.indptr[j]:A.indptr[j + 1]]].tolist())
        aidx.extend(sorted(nb))
        aptr.append(len(aidx))
    return np.array(aptr, dtype=np.int64), np.array(aidx, dtype=np.int32)


def icohp(rho: np.ndarray, A, cols, offsets, orb_offset, orb_count):
    """Connectivity C_IJ = sum_a sum_b rho_{Ia;Jb} A_{Jb;Ia} (Sec. VII, ICOHP),
    summed over the solved columns Jb only, on the atom pattern of A.

    rho is on the pattern layout of the columns (rho[offsets[c] + t] is
    rho_{i_t, cols[c]}). Returns (aptr, aidx, C) with C[aptr[J] + s] = C_{aidx[s], J}.
    Summing C over everything gives Tr(rho A) over the same columns.
    """
    aptr, aidx = atom_pattern(A, orb_offset, orb_count)
    n_atoms = len(orb_offset)
    atom_of = np.repeat(np.arange(n_atoms), np.asarray(orb_count, dtype=np.int64))
    C = np.zeros(len(aidx))
    for c, j in enumerate(np.asarray(cols).tolist()):
        J = int(atom_of[j])
        nbrs = aidx[aptr[J]:aptr[J + 1]].tolist()
        for t, e in enumerate(range(A.indptr[j], A.indptr[j + 1])):
            i = int(A.indices[e])
            s = nbrs.index(int(atom_of[i]))
            C[aptr[J] + s] += rho[offsets[c] + t] * A.data[e]    # A symmetric: A_{j,i} = A_{i,j}
    return aptr, aidx, C
