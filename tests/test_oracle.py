"""Pins of the CPU oracle against what the mathematics fixes (no GPU).

Each test ties an oracle function to something other than itself: the
generalized eigendecomposition closed form (Eq. EQ-EIG-GREEN), hand-derived
inverses of tiny pencils, brute-force adjugate inverses, symmetry
invariants, an independent solver (COCG) and the exact quadrature identity
Tr(rho B) = sum_m sum_k w_k f(e_k) (-1/pi) Im 1/(z_k - lambda_m), which holds
because y_m^T B y_m = 1.
"""

import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import dense, density, krylov
from paper_1609_08377_gb300 import synthetic as syn


@pytest.fixture(scope="module")
def c64():
    return syn.make_system(64, 1.0, 0)


@pytest.fixture(scope="module")
def ch1k():
    return syn.make_system(1000, 1.0 / 3.0, 0)


def _dense_pencil(M, seed, full=True):
    """A small random symmetric A and SPD B with a full pattern."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-3, 3, (M, M))
    A = (A + A.T) / 2
    E = rng.uniform(-1, 1, (M, M))
    E = (E + E.T) / 2
    np.fill_diagonal(E, 0)
    E *= 0.6 / np.abs(E).sum(axis=1).max()
    B = np.eye(M) + E
    return sp.csr_matrix(A), sp.csr_matrix(B)


# ---------------------------------------------------------------------------
# generator structure (inputs the method relies on)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["c64", "ch1k"])
def test_generator_structure(name, request):
    s = request.getfixturevalue(name)
    A, B = s.A, s.B
    assert (A != A.T).nnz == 0 and (B != B.T).nnz == 0
    assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
    assert s.M == int(s.orb_count.astype(int).sum())
    n_c = int((s.species == syn.SPECIES_C).sum())
    assert n_c == int(round(s.n_atoms * (1.0 if name == "c64" else 1 / 3)))
    assert s.M == (s.n_atoms - n_c) + 4 * n_c
    # B: unit diagonal, Gershgorin radius <= 0.8 -> spectrum in [0.2, 1.8]
    assert np.allclose(B.diagonal(), 1.0)
    lb = np.linalg.eigvalsh(B.toarray())
    assert lb.min() >= 0.2 - 1e-12 and lb.max() <= 1.8 + 1e-12
    # minimum-image distances >= 1.0 A
    d = s.pos[:, None, :] - s.pos[None, :, :]
    d -= s.box * np.round(d / s.box)
    r = np.sqrt((d ** 2).sum(-1)) + np.eye(s.n_atoms) * 1e9
    assert r.min() >= syn.R_MIN
    # on-site values and zero same-atom off-diagonals
    Ad = A.toarray()
    for I in range(min(s.n_atoms, 50)):
        o, c = s.orb_offset[I], s.orb_count[I]
        blk = Ad[o:o + c, o:o + c]
        want = syn.ONSITE_C if c == 4 else syn.ONSITE_H
        assert np.allclose(np.diag(blk), want)
        assert np.count_nonzero(blk - np.diag(np.diag(blk))) == 0
    # every stored (I, J) block is a full orbital block: pattern is atom-blocked
    atom = s.atom_of_row()
    rows = np.repeat(np.arange(s.M), np.diff(A.indptr))
    pairs = set(zip(atom[rows].tolist(), atom[A.indices].tolist()))
    assert A.nnz == sum(int(s.orb_count[i]) * int(s.orb_count[j]) for i, j in pairs)


def test_generator_is_seeded():
    a = syn.make_system(64, 1.0, 3)
    b = syn.make_system(64, 1.0, 3)
    c = syn.make_system(64, 1.0, 4)
    assert np.array_equal(a.A.data, b.A.data) and np.array_equal(a.pos, b.pos)
    assert not np.array_equal(a.pos, c.pos)


def test_trapezoid_weights_integrate_linear_exactly():
    eps = syn.energy_grid(16)
    w = syn.trapezoid_weights(eps)
    assert np.isclose(w.sum(), 30.0)
    assert np.isclose(w @ eps, (5.0 ** 2 - 25.0 ** 2) / 2)


# ---------------------------------------------------------------------------
# O1 / O2: the definition and the closed form
# ---------------------------------------------------------------------------

def test_lu_matches_closed_form_c64(c64):
    z = syn.shifts(syn.energy_grid(16), 0.1)
    cols = np.arange(c64.M)
    G1 = dense.green_lu(c64.A, c64.B, z, cols)
    G2 = dense.green_eig(c64.A, c64.B, z, cols)
    assert np.abs(G1 - G2).max() / np.abs(G2).max() < 1e-12


def test_lu_matches_closed_form_ch1k_subset(ch1k):
    z = syn.shifts(syn.energy_grid(64), 0.1)[::16]
    cols = np.array([0, 17, 999, 1998])
    G1 = dense.green_lu(ch1k.A, ch1k.B, z, cols)
    G2 = dense.green_eig(ch1k.A, ch1k.B, z, cols)
    assert np.abs(G1 - G2).max() / np.abs(G2).max() < 1e-12


def test_layout_against_dense_inverse(c64):
    """Element (i, j, k) of the flat layout equals [(z_k B - A)^{-1}]_{ij}."""
    z = syn.shifts(syn.energy_grid(16), 0.1)
    cols = np.array([3, 100, 255])
    G1 = dense.green_lu(c64.A, c64.B, z, cols)
    off = dense.pattern_offsets(c64.A, cols)
    for k in (0, 9):
        inv = np.linalg.inv(z[k] * c64.B.toarray() - c64.A.toarray())
        for c, j in enumerate(cols):
            rows = c64.A.indices[c64.A.indptr[j]:c64.A.indptr[j + 1]]
            assert np.allclose(G1[off[c]:off[c + 1], k], inv[rows, j], rtol=1e-12, atol=1e-14)


def test_green_symmetry_and_conjugation(c64):
    """G(z)^T = G(z) (A, B symmetric) and G(conj z) = conj G(z)."""
    z = np.array([-12.3 + 0.1j, 2.0 + 0.05j])
    cols = np.arange(c64.M)
    G = dense.green_lu(c64.A, c64.B, z, cols)
    Gc = dense.green_lu(c64.A, c64.B, np.conj(z), cols)
    assert np.abs(Gc - np.conj(G)).max() < 1e-12 * np.abs(G).max()
    off = dense.pattern_offsets(c64.A, cols)
    A = c64.A
    lookup = {}
    for j in range(c64.M):
        for t, i in enumerate(A.indices[A.indptr[j]:A.indptr[j + 1]]):
            lookup[(int(i), j)] = off[j] + t
    worst = 0.0
    for (i, j), e in lookup.items():
        worst = max(worst, np.abs(G[e] - G[lookup[(j, i)]]).max())
    assert worst < 1e-12 * np.abs(G).max()


def test_single_carbon_atom():
    """An isolated C atom: B = I, G = diag(1/(z - e_s), 1/(z - e_p) x3)."""
    A = sp.csr_matrix(np.diag(syn.ONSITE_C))
    B = sp.csr_matrix(np.eye(4))
    z = np.array([-19.0 + 0.1j, -10.0 + 0.2j])
    G = dense.green_lu(A, B, z, np.arange(4))
    for k, zk in enumerate(z):
        want = 1.0 / (zk - np.asarray(syn.ONSITE_C))
        assert np.allclose(G[:, k], want, rtol=1e-14)


def test_h2_pair_analytic():
    """2x2 pencil: eigenvalues (e +- t)/(1 +- s); inverse by the 2x2 adjugate."""
    e, t, s = -13.6, -2.1, 0.3
    A = sp.csr_matrix(np.array([[e, t], [t, e]]))
    B = sp.csr_matrix(np.array([[1.0, s], [s, 1.0]]))
    lam, _ = dense.generalized_eigh(A, B)
    assert np.allclose(np.sort(lam), np.sort([(e + t) / (1 + s), (e - t) / (1 - s)]), rtol=1e-14)
    z = np.array([-15.0 + 0.1j, -11.0 + 0.3j])
    G = dense.green_lu(A, B, z, [0, 1])
    for k, zk in enumerate(z):
        a, b = zk - e, zk * s - t          # zB - A = [[a, b], [b, a]]
        det = a * a - b * b
        inv = np.array([[a, -b], [-b, a]]) / det
        assert np.allclose(G[0:2, k], inv[:, 0], rtol=1e-13)
        assert np.allclose(G[2:4, k], inv[:, 1], rtol=1e-13)


def test_identity_overlap_diagonal_hamiltonian():
    """B = I (ordinary shifted equations) with diagonal A: G = diag(1/(z - a_i))."""
    a = np.array([-5.0, -1.0, 0.5, 3.0, 7.0])
    A = sp.csr_matrix(np.diag(a))
    B = sp.csr_matrix(np.eye(5))
    z = np.array([0.1 + 0.1j, -4.0 + 0.05j])
    for fn in (dense.green_lu, dense.green_eig):
        G = fn(A, B, z, np.arange(5))
        for k, zk in enumerate(z):
            assert np.allclose(G[:, k], 1.0 / (zk - a), rtol=1e-14)
    r = krylov.lanczos_column(A, B, 2, z, tol=1e-13, check_every=1)
    assert np.allclose(r.G[:, 0], [1.0 / (z[0] - a[2])], rtol=1e-12)


def _adjugate_inverse(K):
    """Pure-Python inverse of a small complex matrix by cofactors (brute force)."""
    n = len(K)

    def det(m):
        if len(m) == 1:
            return m[0][0]
        return sum(((-1) ** c) * m[0][c] * det([row[:c] + row[c + 1:] for row in m[1:]])
                   for c in range(len(m)))

    d = det(K)
    inv = [[0j] * n for _ in range(n)]
    for i, j in itertools.product(range(n), range(n)):
        minor = [row[:j] + row[j + 1:] for r, row in enumerate(K) if r != i]
        inv[j][i] = ((-1) ** (i + j)) * det(minor) / d
    return inv


def test_bruteforce_tiny_pencil():
    A, B = _dense_pencil(4, seed=11)
    z = np.array([0.3 + 0.2j, -1.7 + 0.05j])
    G = dense.green_lu(A, B, z, np.arange(4))
    Ad, Bd = A.toarray(), B.toarray()
    for k, zk in enumerate(z):
        K = [[complex(zk * Bd[i, j] - Ad[i, j]) for j in range(4)] for i in range(4)]
        inv = np.array(_adjugate_inverse(K))
        assert np.allclose(G[:, k].reshape(4, 4).T, inv, rtol=1e-11, atol=1e-13)


# ---------------------------------------------------------------------------
# O3 / O3': Krylov oracles
# ---------------------------------------------------------------------------

def test_cg_solve_matches_direct(c64):
    rng = np.random.default_rng(5)
    U = rng.standard_normal((c64.M, 3))
    V = krylov.cg_solve(c64.B, U, tol=1e-14)
    assert np.abs(V - np.linalg.solve(c64.B.toarray(), U)).max() < 1e-12


def test_lanczos_matches_lu_c64(c64):
    z = syn.shifts(syn.energy_grid(16), 0.1)
    cols = np.array([0, 77, 200])
    G1 = dense.green_lu(c64.A, c64.B, z, cols)
    zc = [z] * cols.size
    G3, iters, _, conv = krylov.lanczos_columns(c64.A, c64.B, cols, zc, tol=1e-10)
    assert conv.all()
    assert np.abs(G3 - G1).max() / np.abs(G1).max() < 1e-10


def test_lanczos_true_residual(c64):
    """The stopping estimate |y_n| ||u_n|| tracks the true FP64 residual."""
    z = syn.shifts(syn.energy_grid(16), 0.1)
    j = 31
    r = krylov.lanczos_column(c64.A, c64.B, j, z, tol=1e-9, keep_full=True)
    e = np.zeros(c64.M)
    e[j] = 1.0
    for k in range(z.size):
        res = e - (z[k] * c64.B - c64.A) @ r.x_full[:, k]
        assert np.linalg.norm(res) < 1e-8
    assert r.resid.max() <= 1e-9


def test_lanczos_per_column_eta(c64):
    """Shifts with another damping: O3 still equals O1 (z enters only the scalars)."""
    z = syn.shifts(syn.energy_grid(16), 0.2)
    G1 = dense.green_lu(c64.A, c64.B, z, [9])
    r = krylov.lanczos_column(c64.A, c64.B, 9, z, tol=1e-10)
    assert np.abs(r.G - G1).max() / np.abs(G1).max() < 1e-10


def test_cocg_spot_check(c64):
    z = syn.shifts(syn.energy_grid(16), 0.1)
    j, k = 40, 11
    x, _ = krylov.cocg_solve(c64.A, c64.B, j, z[k], tol=1e-11)
    r = krylov.lanczos_column(c64.A, c64.B, j, z, tol=1e-10)
    rows = dense.pattern_rows(c64.A, j)
    assert np.abs(x[rows] - r.G[:, k]).max() / np.abs(x).max() < 1e-8


# ---------------------------------------------------------------------------
# density: Fermi function and the quadrature identities
# ---------------------------------------------------------------------------

def test_fermi_properties():
    mu, kT = -10.0, 0.1
    assert density.fermi(mu, mu, kT) == 0.5
    x = np.linspace(-5, 5, 101)
    f = density.fermi(mu + x, mu, kT)
    assert np.allclose(f + density.fermi(mu - x, mu, kT), 1.0, atol=1e-15)
    with np.errstate(over="raise"):
        ext = density.fermi(np.array([-1e6, 1e6]), mu, kT)
    assert ext[0] == 1.0 and ext[1] == 0.0
    assert np.isclose(density.fermi(mu + kT, mu, kT), 1 / (1 + np.e))


def _quadrature_sum(lam, z, w, f):
    """sum_m sum_k w_k f_k (-1/pi) Im 1/(z_k - lambda_m), per eigenvalue."""
    return (-(1 / np.pi) * np.imag(1.0 / (z[None, :] - lam[:, None])) * (w * f)[None, :]).sum(axis=1)


@pytest.mark.parametrize("n_shifts", [16, 64])
def test_quadrature_identity(c64, n_shifts):
    eps = syn.energy_grid(n_shifts)
    w = syn.trapezoid_weights(eps)
    z = syn.shifts(eps, 0.1)
    mu, kT = -10.0, 0.1
    cols = np.arange(c64.M)
    G = dense.green_lu(c64.A, c64.B, z, cols)
    rho = density.density_from_green(G, eps, w, mu, kT)
    off = dense.pattern_offsets(c64.A, cols)
    lam, _ = dense.generalized_eigh(c64.A, c64.B)
    per = _quadrature_sum(lam, z, w, density.fermi(eps, mu, kT))
    trB = density.trace_with(rho, c64.B, cols, off)
    trA = density.trace_with(rho, c64.A, cols, off)
    assert abs(trB - per.sum()) < 1e-10 * max(1.0, abs(per.sum()))
    assert abs(trA - (lam * per).sum()) < 1e-10 * max(1.0, abs((lam * per).sum()))


def test_sum_rule_fine_grid():
    """Tr(rho B) -> sum_m f(lambda_m) on a fine, wide grid, within a derived bound.

    Per eigenvalue the quadrature of f against the Lorentzian of width eta
    differs from f(lambda) by (a) the Lorentzian mass outside the window,
    (b) the smoothing of f by the Lorentzian, bounded with the Lipschitz
    constant of f near lambda and the tail mass beyond half the distance to
    mu, and (c) the trapezoid error, negligible at spacing eta/8.
    """
    A, B = _dense_pencil(10, seed=2)
    lam, _ = dense.generalized_eigh(A, B)
    mu, kT, eta = float(np.median(lam)) + 0.37, 0.1, 0.004
    lo, hi = lam.min() - 40, lam.max() + 40
    n = int(np.ceil((hi - lo) / (eta / 8))) + 1
    eps = np.linspace(lo, hi, n)
    w = syn.trapezoid_weights(eps)
    z = syn.shifts(eps, eta)
    cols = np.arange(10)
    G = dense.green_eig(A, B, z, cols)
    rho = density.density_from_green(G, eps, w, mu, kT)
    trB = density.trace_with(rho, B, cols, dense.pattern_offsets(A, cols))
    want = density.fermi(lam, mu, kT).sum()
    bound = 0.0
    for l in lam:
        tail = (np.pi / 2 - np.arctan((hi - l) / eta) + np.pi / 2 - np.arctan((l - lo) / eta)) / np.pi
        d = abs(l - mu) / 2
        lip = np.exp(-d / kT) / kT if d > 0 else 1 / (4 * kT)
        lip = min(lip, 1 / (4 * kT))
        smooth = (eta * lip / np.pi) * np.log(1 + (d / eta) ** 2) + (1 - 2 / np.pi * np.arctan(d / eta))
        bound += tail + smooth + 1e-9
    assert abs(trB - want) <= bound
    assert bound < 0.5


# ---------------------------------------------------------------------------
# trace quantities: per-shift traces, chemical potential, ICOHP
# ---------------------------------------------------------------------------

def test_shift_traces_closed_form(c64):
    """Full column set: sum_j (G(z)B)_jj = sum_m 1/(z - lambda_m) and
    sum_j (G(z)A)_jj = sum_m lambda_m/(z - lambda_m) (Eq. EQ-EIG-GREEN)."""
    eps = syn.energy_grid(16)
    z = syn.shifts(eps, 0.1)
    cols = np.arange(c64.M)
    G = dense.green_lu(c64.A, c64.B, z, cols)
    off = dense.pattern_offsets(c64.A, cols)
    lam, _ = dense.generalized_eigh(c64.A, c64.B)
    r = 1.0 / (z[None, :] - lam[:, None])
    sB = density.shift_traces(G, c64.B, cols, off)
    sA = density.shift_traces(G, c64.A, cols, off)
    assert np.allclose(sB, r.sum(axis=0).imag, rtol=1e-10, atol=1e-10)
    assert np.allclose(sA, (lam[:, None] * r).sum(axis=0).imag, rtol=1e-10, atol=1e-10)
    # the count at any mu is the trace of the quadrature density matrix
    w = syn.trapezoid_weights(eps)
    rho = density.density_from_green(G, eps, w, -8.0, 0.3)
    assert np.isclose(density.count_from_traces(sB, eps, w, -8.0, 0.3),
                      density.trace_with(rho, c64.B, cols, off), rtol=1e-12)


def _diag_pencil_green(a, z):
    """G for A = diag(a), B = I on a diagonal pattern: G_ii = 1/(z - a_i)."""
    M = a.size
    A = sp.csr_matrix(np.diag(a))
    B = sp.identity(M, format="csr")
    G = 1.0 / (z[None, :] - a[:, None])
    return A, B, G


def test_find_mu_symmetric_spectrum():
    """Spectrum and grid symmetric about 0, n_elec = half the f = 1 count:
    f(e) + f(-e) = 1 at mu = 0 makes N(0) exactly that half, so mu = 0."""
    a = np.array([-3.0, -1.2, -0.4, 0.4, 1.2, 3.0])
    eps = np.linspace(-6, 6, 241)
    w = syn.trapezoid_weights(eps)
    z = syn.shifts(eps, 0.2)
    A, B, G = _diag_pencil_green(a, z)
    cols = np.arange(a.size)
    s = density.shift_traces(G, B, cols, dense.pattern_offsets(A, cols))
    full = float(-(w @ s) / np.pi)
    mu = density.find_mu(s, eps, w, 0.1, 0.5 * full, -5.0, 5.0)
    assert abs(mu) < 1e-12


def test_find_mu_gap_and_count():
    """A gapped spectrum, a fine grid, small eta and kT: the mu that holds three
    electrons lies inside the gap between the third and fourth level, and the
    count there matches the target."""
    a = np.array([-7.0, -6.5, -5.0, -1.0, 0.5, 2.0])
    eps = np.linspace(-40, 40, 16001)
    w = syn.trapezoid_weights(eps)
    z = syn.shifts(eps, 0.02)
    A, B, G = _diag_pencil_green(a, z)
    cols = np.arange(a.size)
    s = density.shift_traces(G, B, cols, dense.pattern_offsets(A, cols))
    mu = density.find_mu(s, eps, w, 0.05, 3.0, -20.0, 20.0)
    assert -5.0 < mu < -1.0
    assert abs(density.count_from_traces(s, eps, w, mu, 0.05) - 3.0) < 1e-10
    with pytest.raises(ValueError):
        density.find_mu(s, eps, w, 0.05, 7.0, -20.0, 20.0)


def test_icohp_bruteforce_and_energy(c64):
    """C_IJ against dense blocks of the exact density matrix, the sum rule
    sum_IJ C_IJ = Tr(rho A) (Sec. VII), and C_IJ = C_JI for a symmetric rho."""
    eps = syn.energy_grid(16)
    w = syn.trapezoid_weights(eps)
    z = syn.shifts(eps, 0.1)
    mu, kT = -10.0, 0.1
    cols = np.arange(c64.M)
    G = dense.green_lu(c64.A, c64.B, z, cols)
    off = dense.pattern_offsets(c64.A, cols)
    rho = density.density_from_green(G, eps, w, mu, kT)
    aptr, aidx, C = density.icohp(rho, c64.A, cols, off, c64.orb_offset, c64.orb_count)
    # dense rho from the same quadrature, column by column through G = (zB - A)^-1
    Ad = c64.A.toarray()
    Rd = np.zeros_like(Ad)
    coef = w * density.fermi(eps, mu, kT)
    for k in range(eps.size):
        Rd += -(coef[k] / np.pi) * dense.green_dense_full(c64.A, c64.B, z[k]).imag
    oo, oc = c64.orb_offset.astype(int), c64.orb_count.astype(int)
    for J in range(c64.n_atoms):
        sJ = slice(oo[J], oo[J] + oc[J])
        for s in range(aptr[J], aptr[J + 1]):
            I = int(aidx[s])
            sI = slice(oo[I], oo[I] + oc[I])
            want = float((Rd[sI, sJ] * Ad[sJ, sI].T).sum())
            assert abs(C[s] - want) <= 1e-10 * max(1.0, abs(want))
    assert np.isclose(C.sum(), density.trace_with(rho, c64.A, cols, off), rtol=1e-12)
    pos = {(int(aidx[s]), J): s for J in range(c64.n_atoms) for s in range(aptr[J], aptr[J + 1])}
    for (I, J), s in pos.items():
        assert abs(C[s] - C[pos[(J, I)]]) <= 1e-10 * max(1.0, abs(C[s]))


def test_icohp_column_subset_on_ch_mix():
    """Mixed C/H atoms and a column subset: only the atoms of solved columns get
    entries, and the total is Tr(rho A) over those columns."""
    s_ = syn.make_system(40, 0.5, 3)
    eps = syn.energy_grid(8)
    w = syn.trapezoid_weights(eps)
    z = syn.shifts(eps, 0.2)
    cols = syn.column_subset(s_.M, 11, 1)
    G = dense.green_lu(s_.A, s_.B, z, cols)
    off = dense.pattern_offsets(s_.A, cols)
    rho = density.density_from_green(G, eps, w, -10.0, 0.1)
    aptr, aidx, C = density.icohp(rho, s_.A, cols, off, s_.orb_offset, s_.orb_count)
    atoms = set(s_.atom_of_row()[cols].tolist())
    for J in range(s_.n_atoms):
        if J not in atoms:
            assert not C[aptr[J]:aptr[J + 1]].any()
    assert np.isclose(C.sum(), density.trace_with(rho, s_.A, cols, off), rtol=1e-12)
