"""Parity at the workload size of the 1,000-atom pencil: every column against
dense LU (O1, the definition G = (z B - A)^-1 of Eq. EQ-SHIFT-EQ-J). The
larger workloads are checked against stored oracle columns in
test_gpu_golden.py."""

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
