"""Parity at the workload sizes: every column of the 1,000-atom pencil against
dense LU, and a property that holds at any size on the 1,000,000-atom pencil
(G(z)^T = G(z) for symmetric A and B: G_ij from column j equals G_ji from
column i), where the oracle cannot finish."""

import numpy as np
import pytest

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


def test_ch1k_all_columns_fp64(gsk):
    """Plain FP64, all 1,999 columns, 64 shifts, tol 1e-8 (the 1,000-atom workload)."""
    s = syn.make_system(1000, 1.0 / 3.0, 0)
    z = syn.shifts(syn.energy_grid(64), 0.1)
    cols = np.arange(s.M, dtype=np.int32)
    solver = gsk.from_system(s)
    off = solver.pattern_offsets(cols)
    G = torch.zeros(int(off[-1]) * 64, dtype=torch.complex128, device="cuda")
    it, st, rs = solver.solve(z, cols, G, precision="fp64", tol=1e-8)
    torch.cuda.synchronize()
    assert (st == gsk.GSK_CONVERGED).all()
    R = dense.green_lu(s.A, s.B, z, cols)
    Gh = G.cpu().numpy().reshape(int(off[-1]), 64)
    assert np.abs(Gh - R).max() / np.abs(R).max() <= 1e-8


def test_ch1m_symmetry(gsk):
    """1,000,000 atoms (M ~ 2e6): G_ij(z) from column j equals G_ji(z) from column i."""
    s = syn.make_system(1000000, 1.0 / 3.0, 0)
    A = s.A
    i = int(syn.column_subset(s.M, 1, 0)[0])
    nb = A.indices[A.indptr[i]:A.indptr[i + 1]]
    j = int(nb[nb != i][len(nb) // 2 - 1])
    solver = gsk.from_system(s)
    cols = np.array([i, j], dtype=np.int32)
    z = syn.shifts(syn.energy_grid(16), 0.2)
    off = solver.pattern_offsets(cols)
    G = torch.zeros(int(off[-1]) * 16, dtype=torch.complex128, device="cuda")
    it, st, _ = solver.solve(z, cols, G, precision="mixed_df", tol=1e-8, batch_w=32)
    torch.cuda.synchronize()
    assert (st == gsk.GSK_CONVERGED).all()
    Gh = G.cpu().numpy().reshape(int(off[-1]), 16)
    rows_i = A.indices[A.indptr[i]:A.indptr[i + 1]]
    rows_j = A.indices[A.indptr[j]:A.indptr[j + 1]]
    g_ji = Gh[off[0] + int(np.nonzero(rows_i == j)[0][0])]     # row j of column i
    g_ij = Gh[off[1] + int(np.nonzero(rows_j == i)[0][0])]     # row i of column j
    scale = np.abs(Gh).max()
    assert np.abs(g_ij - g_ji).max() <= 1e-8 * scale
