"""Seeded synthetic tight-binding-like pencils (A, B) standing in for the paper's
PPE-polymer and diamond structures, which are not available.

This module only builds INPUTS: atom positions, species, the orbital-block map,
the sparse matrices A (Hamiltonian) and B (overlap), the shift grid, the
quadrature weights of the energy grid, per-column damping and column subsets.
It holds none of the solver's arithmetic, so both the CUDA path and the CPU
oracle may use it.

Physical ingredients taken from the paper (Sec. II-C): every basis index is an
(atom, orbital) pair; H carries one s orbital and C carries s, px, py, pz, so
M = N_H + 4 N_C; matrix elements between atoms farther apart than a cutoff are
dropped, which makes A and B sparse with an atom-block pattern; the structures
are disordered and periodic (Sec. IV-A).

Recipe (all distances in angstrom, energies in eV):
  * atoms are placed by random sequential addition in a periodic cube at
    0.1 atoms / A^3; a candidate closer than 1.0 A (minimum image) to an atom
    already placed is rejected;
  * a fraction of the atoms is C (4 orbitals), the rest H (1 orbital);
    species are assigned by a seeded permutation after placement;
  * A: on-site s = -19.4 (C), p = -10.7 (C), s = -13.6 (H); same-atom
    off-diagonal elements are 0; for atom pairs within r_cut = 5 A
    A_{Ia,Jb} = t_ab * exp(-(r - 1.5) / 0.6), summed over all periodic images
    within the cutoff, with seeded symmetric coupling tables t in [-3, 3];
  * B: identity diagonal; off-diagonal 0.25 * s_ab * exp(-(r - 1.0) / 0.8) with
    seeded tables s in [-1, 1]; every off-diagonal element is then multiplied by
    one global factor c = min(1, 0.8 / max_i sum_{j != i} |B_ij|) so that the
    Gershgorin bounds put the spectrum of B in [0.2, 1.8] (B is SPD);
  * the block pattern is every orbital pair of every atom pair within the
    cutoff, including each atom's own diagonal block (stored explicitly, zeros
    included); B has the same pattern as A.

Seeded draw order (numpy.random.default_rng(seed)): coupling tables
(t_CC upper triangle row-major, t_CH, t_HH, s_CC upper triangle, s_CH, s_HH),
then positions, then the species permutation.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

DENSITY = 0.1        # atoms per A^3
R_MIN = 1.0          # rejection distance, A
R_CUT = 5.0          # cutoff, A
ONSITE_C = (-19.4, -10.7, -10.7, -10.7)
ONSITE_H = (-13.6,)
T_RANGE = 3.0
S_RANGE = 1.0
A_R0, A_DECAY = 1.5, 0.6
B_PREF, B_R0, B_DECAY = 0.25, 1.0, 0.8
B_GERSHGORIN_RADIUS = 0.8

SPECIES_H = 0
SPECIES_C = 1


@dataclasses.dataclass
class System:
    """One synthetic pencil and its orbital-block map (original atom order)."""

    n_atoms: int
    box: float
    pos: np.ndarray           # (N, 3) float64
    species: np.ndarray       # (N,) int8, SPECIES_H or SPECIES_C
    orb_count: np.ndarray     # (N,) int8, 1 or 4
    orb_offset: np.ndarray    # (N,) int32, first basis index of each atom
    A: sp.csr_matrix          # (M, M) float64, explicit pattern
    B: sp.csr_matrix          # (M, M) float64, same pattern as A
    b_scale: float            # global factor applied to B's off-diagonals
    tables: dict

    @property
    def M(self) -> int:
        return int(self.A.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.A.nnz)

    def atom_of_row(self) -> np.ndarray:
        return np.repeat(np.arange(self.n_atoms, dtype=np.int32), self.orb_count.astype(np.int64))


def _draw_tables(rng: np.random.Generator) -> dict:
    def sym4(lo_hi: float) -> np.ndarray:
        upper = rng.uniform(-lo_hi, lo_hi, size=10)
        t = np.zeros((4, 4))
        t[np.triu_indices(4)] = upper
        return t + np.triu(t, 1).T

    t_cc = sym4(T_RANGE)
    t_ch = rng.uniform(-T_RANGE, T_RANGE, size=4)
    t_hh = rng.uniform(-T_RANGE, T_RANGE, size=1)
    s_cc = sym4(S_RANGE)
    s_ch = rng.uniform(-S_RANGE, S_RANGE, size=4)
    s_hh = rng.uniform(-S_RANGE, S_RANGE, size=1)
    return {"t_cc": t_cc, "t_ch": t_ch, "t_hh": t_hh, "s_cc": s_cc, "s_ch": s_ch, "s_hh": s_hh}


def _species_table(cc: np.ndarray, ch: np.ndarray, hh: np.ndarray) -> np.ndarray:
    """tab[species_I, species_J, a, b]: coupling between orbital a of I and b of J."""
    tab = np.zeros((2, 2, 4, 4))
    tab[SPECIES_C, SPECIES_C] = cc
    tab[SPECIES_H, SPECIES_C, 0, :] = ch
    tab[SPECIES_C, SPECIES_H, :, 0] = ch
    tab[SPECIES_H, SPECIES_H, 0, 0] = hh[0]
    return tab


def _place_atoms(rng: np.random.Generator, n: int, box: float) -> np.ndarray:
    """Random sequential addition with minimum-image rejection at R_MIN.

    Candidates are drawn from the generator in order; a candidate is accepted
    when no previously accepted atom lies within R_MIN. Work proceeds in chunks
    but the result equals the one-at-a-time procedure on the same stream.
    """
    ncell = max(1, int(box // R_MIN))
    cell = box / ncell
    cap = 16
    grid = np.full((ncell, ncell, ncell, cap), -1, dtype=np.int64)
    fill = np.zeros((ncell, ncell, ncell), dtype=np.int64)
    pos = np.empty((n, 3))
    count = 0
    offs = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)])
    while count < n:
        need = n - count
        chunk = int(min(max(2 * need + 64, 256), 262144))
        cand = rng.uniform(0.0, box, size=(chunk, 3))
        ci = np.minimum((cand / cell).astype(np.int64), ncell - 1)
        ok = np.ones(chunk, dtype=bool)
        # against atoms accepted in earlier chunks
        for o in offs:
            nc = (ci + o) % ncell
            slots = grid[nc[:, 0], nc[:, 1], nc[:, 2]]          # (chunk, cap)
            valid = slots >= 0
            if not valid.any():
                continue
            other = pos[np.where(valid, slots, 0)]               # (chunk, cap, 3)
            d = other - cand[:, None, :]
            d -= box * np.round(d / box)
            r2 = np.einsum("ijk,ijk->ij", d, d)
            ok &= ~np.any(valid & (r2 < R_MIN * R_MIN), axis=1)
        # conflicts inside the chunk, resolved in draw order
        idx = np.nonzero(ok)[0]
        if idx.size > 1:
            from scipy.spatial import cKDTree

            sub = np.mod(cand[idx], box)
            tree = cKDTree(sub, boxsize=box)
            pairs = tree.query_pairs(R_MIN * (1 + 1e-9), output_type="ndarray")
            if pairs.size:
                # exact check with the same arithmetic as above
                d = sub[pairs[:, 1]] - sub[pairs[:, 0]]
                d -= box * np.round(d / box)
                close = np.einsum("ij,ij->i", d, d) < R_MIN * R_MIN
                pairs = pairs[close]
            if pairs.size:
                lo = np.minimum(pairs[:, 0], pairs[:, 1])
                hi = np.maximum(pairs[:, 0], pairs[:, 1])
                order = np.argsort(hi, kind="stable")
                lo, hi = lo[order], hi[order]
                accepted = np.ones(idx.size, dtype=bool)
                for a, b in zip(lo.tolist(), hi.tolist()):
                    if accepted[a] and accepted[b]:
                        accepted[b] = False
                idx = idx[accepted]
        idx = idx[:need]
        for k in idx.tolist():
            c = ci[k]
            f = fill[c[0], c[1], c[2]]
            assert f < cap, "cell capacity exceeded"
            grid[c[0], c[1], c[2], f] = count
            fill[c[0], c[1], c[2]] += 1
            pos[count] = cand[k]
            count += 1
    return pos


def _pairs_bruteforce(pos: np.ndarray, box: float, rcut: float):
    """All (I, J, r) with r <= rcut over periodic images, I != J or a nonzero image."""
    n = pos.shape[0]
    k = int(math.ceil(rcut / box))
    shifts = np.array([(a, b, c) for a in range(-k, k + 1) for b in range(-k, k + 1)
                       for c in range(-k, k + 1)], dtype=np.float64) * box
    out_i, out_j, out_r = [], [], []
    for i in range(n):
        d = pos[None, :, :] + shifts[:, None, :] - pos[i][None, None, :]   # (S, N, 3)
        r = np.sqrt(np.einsum("sjk,sjk->sj", d, d))
        sel = r <= rcut
        sel[shifts.shape[0] // 2, i] = False        # the atom itself, zero image
        s_idx, j_idx = np.nonzero(sel)
        if np.any(j_idx == i):
            raise ValueError("box smaller than the cutoff: self-images are not supported")
        out_i.append(np.full(j_idx.size, i, dtype=np.int64))
        out_j.append(j_idx.astype(np.int64))
        out_r.append(r[s_idx, j_idx])
    return np.concatenate(out_i), np.concatenate(out_j), np.concatenate(out_r)


def _pairs_kdtree(pos: np.ndarray, box: float, rcut: float):
    """Directed pairs within rcut for boxes larger than 2*rcut (one image per pair)."""
    from scipy.spatial import cKDTree

    assert box > 2 * rcut
    p = np.mod(pos, box)
    tree = cKDTree(p, boxsize=box)
    pr = tree.query_pairs(rcut * (1 + 1e-12), output_type="ndarray").astype(np.int64)
    d = p[pr[:, 1]] - p[pr[:, 0]]
    d -= box * np.round(d / box)
    r = np.sqrt(np.einsum("ij,ij->i", d, d))
    keep = r <= rcut
    pr, r = pr[keep], r[keep]
    i = np.concatenate([pr[:, 0], pr[:, 1]])
    j = np.concatenate([pr[:, 1], pr[:, 0]])
    return i, j, np.concatenate([r, r])


def _assemble(n, orb_count, orb_offset, species, pi, pj, gA, gB, tab_a, tab_b, onsite):
    """CSR A and B from directed atom pairs (self pairs included) with radial sums."""
    order = np.lexsort((pj, pi))
    pi, pj, gA, gB = pi[order], pj[order], gA[order], gB[order]
    oc = orb_count.astype(np.int64)
    ncols_pair = oc[pj]
    # row length of every orbital row of atom I: sum of orb_J over neighbours J
    row_len_atom = np.bincount(pi, weights=ncols_pair, minlength=n).astype(np.int64)
    M = int(oc.sum())
    row_atom = np.repeat(np.arange(n), oc)
    indptr = np.zeros(M + 1, dtype=np.int64)
    np.cumsum(row_len_atom[row_atom], out=indptr[1:])
    # column offset of pair p inside the rows of atom pi[p]
    first = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(pi, minlength=n), out=first[1:])
    csum = np.cumsum(ncols_pair) - ncols_pair
    within = csum - csum[first[pi]]
    nnz = int(indptr[-1])
    indices = np.empty(nnz, dtype=np.int32)
    da = np.empty(nnz)
    db = np.empty(nnz)
    self_pair = pi == pj
    si, sj = species[pi].astype(np.int64), species[pj].astype(np.int64)
    for a in range(4):
        ma = oc[pi] > a
        for b in range(4):
            m = ma & (oc[pj] > b)
            if not m.any():
                continue
            row = orb_offset[pi[m]].astype(np.int64) + a
            pos = indptr[row] + within[m] + b
            indices[pos] = orb_offset[pj[m]] + b
            va = tab_a[si[m], sj[m], a, b] * gA[m]
            vb = tab_b[si[m], sj[m], a, b] * gB[m]
            s = self_pair[m]
            if a == b:
                va = np.where(s, onsite[si[m], a], va)
                vb = np.where(s, 1.0, vb)
            else:
                va = np.where(s, 0.0, va)
                vb = np.where(s, 0.0, vb)
            da[pos] = va
            db[pos] = vb
    A = sp.csr_matrix((da, indices, indptr), shape=(M, M))
    B = sp.csr_matrix((db, indices.copy(), indptr.copy()), shape=(M, M))
    return A, B


def make_system(n_atoms: int, c_fraction: float, seed: int, rcut: float = R_CUT,
                density: float = DENSITY) -> System:
    """Build the seeded pencil for n_atoms atoms with the given C fraction."""
    rng = np.random.default_rng(seed)
    tables = _draw_tables(rng)
    box = (n_atoms / density) ** (1.0 / 3.0)
    pos = _place_atoms(rng, n_atoms, box)
    n_c = int(round(n_atoms * c_fraction))
    species = np.full(n_atoms, SPECIES_H, dtype=np.int8)
    species[rng.permutation(n_atoms)[:n_c]] = SPECIES_C
    orb_count = np.where(species == SPECIES_C, 4, 1).astype(np.int8)
    orb_offset = np.zeros(n_atoms, dtype=np.int32)
    orb_offset[1:] = np.cumsum(orb_count.astype(np.int64))[:-1]

    if box > 2 * rcut:
        pi, pj, r = _pairs_kdtree(pos, box, rcut)
    else:
        pi, pj, r = _pairs_bruteforce(pos, box, rcut)
    fa = np.exp(-(r - A_R0) / A_DECAY)
    fb = B_PREF * np.exp(-(r - B_R0) / B_DECAY)
    # sum the periodic images of each unordered pair {I, J} once (in a fixed
    # order), then emit both directions, so that A and B are exactly symmetric
    lo, hi = np.minimum(pi, pj), np.maximum(pi, pj)
    fwd = pi < pj
    key = lo[fwd] * n_atoms + hi[fwd]
    order = np.lexsort((r[fwd], key))
    key, fa, fb = key[order], fa[fwd][order], fb[fwd][order]
    uk, inv = np.unique(key, return_inverse=True)
    gA = np.bincount(inv, weights=fa)
    gB = np.bincount(inv, weights=fb)
    ui, uj = uk // n_atoms, uk % n_atoms
    selfs = np.arange(n_atoms, dtype=np.int64)
    pi = np.concatenate([ui, uj, selfs])
    pj = np.concatenate([uj, ui, selfs])
    gA = np.concatenate([gA, gA, np.zeros(n_atoms)])
    gB = np.concatenate([gB, gB, np.zeros(n_atoms)])

    tab_a = _species_table(tables["t_cc"], tables["t_ch"], tables["t_hh"])
    tab_b = _species_table(tables["s_cc"], tables["s_ch"], tables["s_hh"])
    onsite = np.zeros((2, 4))
    onsite[SPECIES_C] = ONSITE_C
    onsite[SPECIES_H, 0] = ONSITE_H[0]
    A, B = _assemble(n_atoms, orb_count, orb_offset, species, pi, pj, gA, gB, tab_a, tab_b, onsite)

    # global rescale of B's off-diagonal part (Gershgorin lower bound >= 0.2)
    rows = np.repeat(np.arange(B.shape[0]), np.diff(B.indptr))
    offd = rows != B.indices
    radius = np.bincount(rows[offd], weights=np.abs(B.data[offd]), minlength=B.shape[0])
    rmax = float(radius.max()) if radius.size else 0.0
    c = 1.0 if rmax <= B_GERSHGORIN_RADIUS else B_GERSHGORIN_RADIUS / rmax
    B.data[offd] *= c
    return System(n_atoms=n_atoms, box=box, pos=pos, species=species, orb_count=orb_count,
                  orb_offset=orb_offset, A=A, B=B, b_scale=c, tables=tables)


# ---------------------------------------------------------------------------
# shifts, energy grid, per-column damping and column subsets
# ---------------------------------------------------------------------------

def energy_grid(n_shifts: int, lo: float = -25.0, hi: float = 5.0) -> np.ndarray:
    """Evenly spaced real parts eps_k of the shifts on [lo, hi]."""
    return np.linspace(lo, hi, n_shifts)


def trapezoid_weights(eps: np.ndarray) -> np.ndarray:
    """Trapezoid-rule weights of an evenly spaced grid (half weight at both ends)."""
    n = eps.size
    if n == 1:
        return np.zeros(1)
    h = (eps[-1] - eps[0]) / (n - 1)
    w = np.full(n, h)
    w[0] = w[-1] = h / 2
    return w


def shifts(eps: np.ndarray, eta: float) -> np.ndarray:
    return eps.astype(np.complex128) + 1j * eta


def column_subset(M: int, n_cols: int, seed: int) -> np.ndarray:
    """Seeded uniform sample of n_cols distinct columns (sorted), or all columns."""
    if n_cols >= M:
        return np.arange(M, dtype=np.int32)
    rng = np.random.default_rng(seed + 7919)
    return np.sort(rng.choice(M, size=n_cols, replace=False)).astype(np.int32)


def eta_per_column(n_cols: int, seed: int, choices=(0.05, 0.1, 0.2)) -> np.ndarray:
    rng = np.random.default_rng(seed + 104729)
    return np.asarray(choices, dtype=np.float64)[rng.integers(0, len(choices), size=n_cols)]


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n_atoms: int
    c_fraction: float
    n_shifts: int
    n_cols: int | None      # None: all columns
    eta: float | None       # None: per-column eta from {0.05, 0.1, 0.2}
    tol: float
    mu: float = -10.0
    kT: float = 0.1


WORKLOADS = {
    "c64": Workload("c64", 64, 1.0, 16, None, 0.1, 1e-10),
    "ch1k": Workload("ch1k", 1000, 1.0 / 3.0, 64, None, 0.1, 1e-8),
    "ch20k": Workload("ch20k", 20000, 1.0 / 3.0, 128, 8192, None, 1e-8),
    "ch100k": Workload("ch100k", 100000, 1.0 / 3.0, 128, 16384, None, 1e-8),
    "ch1m": Workload("ch1m", 1000000, 1.0 / 3.0, 64, 65536, None, 1e-8),
}
