"""Reference of the scheduler's per-column features (plain NumPy definitions).

Test infrastructure only (see the package docstring).

For basis column j = (atom J, orbital a) with damping eta (the imaginary part
of the column's shifts), the 16 raw features are:
  0 log(eta)                       8  A_jj / 10
  1 0.1 / eta                      9  sum_{i != j} |A_ij| / 10
  2 entries of row j / 100        10  sum_{i != j} |B_ij|
  3 neighbour atoms of J / 50     11  sqrt(sum_{i != j} A_ij^2) / 10
  4 4-orbital neighbours / 20     12  A_jj^2 / 100
  5 1-orbital neighbours / 40     13  B_jj
  6 1 if J has 4 orbitals         14  log(1 + sum_i |A_ij|)
  7 a / 3                         15  1
"Neighbour atoms" are the atoms other than J with at least one stored entry in
row j's atom block row. The model sees each feature standardised by the mean
and standard deviation of its training set.
"""

from __future__ import annotations

import numpy as np


def raw_features(A, B, orb_offset, orb_count, cols, eta) -> np.ndarray:
    M = A.shape[0]
    n_atoms = len(orb_offset)
    atom = np.repeat(np.arange(n_atoms), np.asarray(orb_count, dtype=np.int64))
    out = np.zeros((len(cols), 16))
    for c, j in enumerate(np.asarray(cols).tolist()):
        J = int(atom[j])
        a = j - int(orb_offset[J])
        lo, hi = A.indptr[j], A.indptr[j + 1]
        idx = A.indices[lo:hi]
        av = A.data[lo:hi]
        bv = B.data[lo:hi]
        off = idx != j
        # neighbour atoms from the whole atom block row of J
        nb = set()
        for r in range(int(orb_offset[J]), int(orb_offset[J]) + int(orb_count[J])):
            nb.update(atom[A.indices[A.indptr[r]:A.indptr[r + 1]]].tolist())
        nb.discard(J)
        n4 = sum(1 for I in nb if orb_count[I] == 4)
        n1 = len(nb) - n4
        ajj = float(av[~off].sum())
        bjj = float(bv[~off].sum())
        e = float(eta[c])
        out[c] = [np.log(e), 0.1 / e, (hi - lo) / 100.0, len(nb) / 50.0, n4 / 20.0, n1 / 40.0,
                  1.0 if orb_count[J] == 4 else 0.0, a / 3.0, ajj / 10.0, np.abs(av[off]).sum() / 10.0,
                  np.abs(bv[off]).sum(), np.sqrt((av[off] ** 2).sum()) / 10.0, ajj * ajj / 100.0, bjj,
                  np.log1p(np.abs(av).sum()), 1.0]
    return out


def standardise(F: np.ndarray, mean: np.ndarray, std: np.ndarray) -> np.ndarray:
    return (F - mean) / std
