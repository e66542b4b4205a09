"""Edge cases of the CUDA path (through the C ABI) against closed forms and the oracle."""

import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dense  # noqa: E402
from paper_1609_08377_gb300 import synthetic as syn  # noqa: E402


@pytest.fixture(scope="module")
def gsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_08377_gb300 import gsk as g
    return g


def _solve(gsk, solver, z, cols, **kw):
    off = solver.pattern_offsets(cols)
    G = torch.zeros(max(1, int(off[-1]) * len(z)), dtype=torch.complex128, device="cuda")
    it, st, rs = solver.solve(z, cols, G, **kw)
    torch.cuda.synchronize()
    return G.cpu().numpy()[: int(off[-1]) * len(z)].reshape(int(off[-1]), len(z)), it, st, rs


def _full_pattern(M):
    idx = np.tile(np.arange(M), M)
    ptr = np.arange(0, M * M + 1, M)
    return idx, ptr


def test_empty_column_set(gsk):
    s = syn.make_system(64, 1.0, 0)
    solver = gsk.from_system(s)
    z = syn.shifts(syn.energy_grid(4), 0.1)
    G = torch.zeros(1, dtype=torch.complex128, device="cuda")
    it, st, rs = solver.solve(z, np.zeros(0, dtype=np.int32), G)
    assert it.size == 0 and st.size == 0


def test_maximum_shift_count(gsk):
    s = syn.make_system(64, 1.0, 0)
    solver = gsk.from_system(s)
    eps = syn.energy_grid(1024)
    z = syn.shifts(eps, 0.2)
    cols = np.array([0, 131])
    G, it, st, _ = _solve(gsk, solver, z, cols, precision="fp64", tol=1e-10)
    assert (st == gsk.GSK_CONVERGED).all()
    R = dense.green_lu(s.A, s.B, z[::64], cols)
    assert np.abs(G[:, ::64] - R).max() <= 1e-8 * np.abs(R).max()
    with pytest.raises(gsk.GskError):
        solver.solve(syn.shifts(syn.energy_grid(1025), 0.2), cols, torch.zeros(10 ** 6, dtype=torch.complex128,
                                                                                device="cuda"))


def test_isolated_atom_invariant_subspace(gsk):
    """One C atom: e_j spans an invariant subspace, the solve ends after one step with G exact."""
    onsite = np.asarray(syn.ONSITE_C)
    idx, ptr = _full_pattern(4)
    A = sp.csr_matrix((np.diag(onsite).ravel(), idx, ptr), shape=(4, 4))
    B = sp.csr_matrix((np.eye(4).ravel(), idx, ptr), shape=(4, 4))
    solver = gsk.Solver(A, B, [0], [4])
    z = np.array([-19.0 + 0.1j, -10.0 + 0.2j, 3.0 + 0.05j])
    for prec in ("fp64", "mixed", "mixed_df"):
        G, it, st, _ = _solve(gsk, solver, z, np.arange(4), precision=prec, tol=1e-12)
        assert (st == gsk.GSK_CONVERGED).all() and (it == 1).all()
        for j in range(4):
            want = np.zeros((4, 3), dtype=complex)
            want[j] = 1.0 / (z - onsite[j])
            assert np.allclose(G[4 * j:4 * j + 4], want, rtol=1e-12, atol=1e-15)


def test_h2_pair_closed_form(gsk):
    """Two H atoms: the 2x2 pencil's inverse is written out by hand."""
    e, t, s_ = -13.6, -2.1, 0.3
    idx, ptr = _full_pattern(2)
    A = sp.csr_matrix((np.array([e, t, t, e]), idx, ptr), shape=(2, 2))
    B = sp.csr_matrix((np.array([1.0, s_, s_, 1.0]), idx, ptr), shape=(2, 2))
    solver = gsk.Solver(A, B, [0, 1], [1, 1])
    z = np.array([-15.0 + 0.1j, -11.0 + 0.3j, -9.0 + 0.05j])
    G, it, st, _ = _solve(gsk, solver, z, np.array([0, 1]), precision="fp64", tol=1e-13)
    assert (st == gsk.GSK_CONVERGED).all()
    for k, zk in enumerate(z):
        a, b = zk - e, zk * s_ - t
        det = a * a - b * b
        assert np.allclose(G[0:2, k], [a / det, -b / det], rtol=1e-11)
        assert np.allclose(G[2:4, k], [-b / det, a / det], rtol=1e-11)


def test_chain_of_hydrogens_padding(gsk):
    """Three H atoms in a line: 1-orbital rows with 1-orbital neighbours use the
    padded four-wide groups of the block layout; compare with dense LU."""
    A = np.array([[-13.6, -1.0, 0.0], [-1.0, -13.6, -0.7], [0.0, -0.7, -13.6]])
    B = np.array([[1.0, 0.2, 0.0], [0.2, 1.0, 0.1], [0.0, 0.1, 1.0]])
    pat = np.abs(A) > 0
    As = sp.csr_matrix(np.where(pat, A, 0.0))
    Bs = sp.csr_matrix((np.where(pat, B, 0.0)[pat], As.indices, As.indptr), shape=(3, 3))
    solver = gsk.Solver(As, Bs, [0, 1, 2], [1, 1, 1])
    z = syn.shifts(np.linspace(-16, -11, 7), 0.1)
    G, it, st, _ = _solve(gsk, solver, z, np.arange(3), precision="mixed_df", tol=1e-12)
    R = dense.green_lu(As, Bs, z, np.arange(3))
    assert np.abs(G - R).max() <= 1e-10 * np.abs(R).max()


def test_step_cap_and_status_codes(gsk):
    """max_iter too small: every column reports GSK_NOT_CONVERGED with its step count."""
    s = syn.make_system(64, 1.0, 0)
    solver = gsk.from_system(s)
    z = syn.shifts(syn.energy_grid(8), 0.05)
    G, it, st, rs = _solve(gsk, solver, z, np.arange(40), precision="mixed_df", tol=1e-10, max_iter=25)
    assert (st == gsk.GSK_NOT_CONVERGED).all() and (it == 25).all() and (rs > 1e-10).all()
