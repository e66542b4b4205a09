"""Real-space projection of one column's problem (Sec. III-B, the technique
that reduces each column to a matrix of size M' = 200-400).

Test infrastructure only (see the package docstring).

For column j of atom J the region is the set of atoms within the distance of
J's kappa-th nearest atom (J itself counted, distances by the minimum-image
convention in a periodic box, ties kept), so it holds kappa atoms or more.
The pencil is restricted to the region's orbitals (the same restriction for
A and for B) and column j of the restricted pencil is solved by the multiple
Arnoldi projection. rho is reported on the full pattern P(j) of A, with zero
for the entries whose row lies outside the region.
"""

from __future__ import annotations

import numpy as np

from . import marnoldi


def min_image_dist2(pos: np.ndarray, J: int, box) -> np.ndarray:
    """Squared distances from atom J to every atom; box = (Lx, Ly, Lz) for
    periodic boundaries or None."""
    d = pos - pos[J]
    if box is not None:
        L = np.asarray(box, dtype=np.float64)
        d = d - L * np.round(d / L)
    return (d * d).sum(axis=1)


def region_atoms(pos: np.ndarray, J: int, kappa: int, box) -> np.ndarray:
    """Atoms within the distance of J's kappa-th nearest atom (ascending index)."""
    d2 = min_image_dist2(pos, J, box)
    k = min(kappa, d2.size)
    cut = np.sort(d2)[k - 1]
    return np.nonzero(d2 <= cut)[0]


def projected_pencil(A, B, orb_offset, orb_count, atoms):
    """(A', B', rows): the pencil restricted to the orbitals of `atoms`, and
    the global row of each local row (ascending)."""
    oo = np.asarray(orb_offset, dtype=np.int64)
    oc = np.asarray(orb_count, dtype=np.int64)
    rows = np.concatenate([np.arange(oo[a], oo[a] + oc[a]) for a in np.sort(atoms)])
    Ap = A[rows][:, rows].tocsr()
    Bp = B[rows][:, rows].tocsr()
    Ap.sort_indices()
    Bp.sort_indices()
    return Ap, Bp, rows


def projected_marnoldi_column(A, B, orb_offset, orb_count, pos, box, j: int, kappa: int, nu: int,
                              mu: float = 0.0, kT: float = 0.1):
    """Multiple Arnoldi on the projected pencil of column j. Returns a dict:
    rho on P(j) of the full A (zeros outside the region), eps / w / q of the
    projected problem, the region's atoms and its number of orbitals."""
    atom_of = np.repeat(np.arange(len(orb_offset)), np.asarray(orb_count, dtype=np.int64))
    atoms = region_atoms(pos, int(atom_of[j]), kappa, box)
    Ap, Bp, rows = projected_pencil(A, B, orb_offset, orb_count, atoms)
    jl = int(np.nonzero(rows == j)[0][0])
    o = marnoldi.marnoldi_column(Ap, Bp, jl, nu, mu=mu, kT=kT)
    prow = A.indices[A.indptr[j]:A.indptr[j + 1]]
    lrow = rows[Ap.indices[Ap.indptr[jl]:Ap.indptr[jl + 1]]]     # global rows of the local pattern
    where = {int(r): t for t, r in enumerate(lrow.tolist())}
    rho = np.array([o["rho"][where[int(i)]] if int(i) in where else 0.0 for i in prow])
    return {"rho": rho, "eps": o["eps"], "w": o["w"], "q": o["q"], "atoms": atoms, "M_local": rows.size}
