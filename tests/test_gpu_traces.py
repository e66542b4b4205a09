"""Trace quantities through the C ABI against the oracle: per-shift traces,
the chemical potential for an electron count, and the ICOHP connectivity
C_IJ (Sec. II, Eq. TRACE-X; Sec. VII).

The CUDA path gets the oracle's G (dense LU, uploaded) or the oracle's rho,
so these tests check the trace kernels alone; the solver's own G is checked
elsewhere.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import dense, density  # noqa: E402
from paper_1609_08377_gb300 import synthetic as syn  # noqa: E402


@pytest.fixture(scope="module")
def gsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_08377_gb300 import gsk as g
    return g


def _case(n_atoms, c_frac, seed, n_shifts, n_cols=None, eta=0.1):
    s = syn.make_system(n_atoms, c_frac, seed)
    cols = np.arange(s.M, dtype=np.int32) if n_cols is None else syn.column_subset(s.M, n_cols, seed)
    eps = syn.energy_grid(n_shifts)
    w = syn.trapezoid_weights(eps)
    z = syn.shifts(eps, eta)
    G = dense.green_lu(s.A, s.B, z, cols)
    off = dense.pattern_offsets(s.A, cols)
    return s, cols, eps, w, z, G, off


def _dev(G):
    return torch.from_numpy(np.ascontiguousarray(G)).to("cuda")


@pytest.mark.parametrize("which", [0, 1])
def test_shift_trace_matches_oracle(gsk, which):
    """64 C atoms, all columns, 40 shifts (two shift tiles, ragged second)."""
    s, cols, eps, w, z, G, off = _case(64, 1.0, 0, 40)
    solver = gsk.from_system(s)
    got = solver.shift_trace(cols, eps.size, _dev(G), which)
    X = s.A if which == 0 else s.B
    want = density.shift_traces(G, X, cols, off)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    solver.close()


def test_shift_trace_subset_and_empty(gsk):
    """C/H mix, a column subset; an empty column set gives zeros."""
    s, cols, eps, w, z, G, off = _case(300, 1.0 / 3.0, 2, 16, n_cols=37)
    solver = gsk.from_system(s)
    got = solver.shift_trace(cols, 16, _dev(G), 1)
    want = density.shift_traces(G, s.B, cols, off)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    empty = solver.shift_trace(np.zeros(0, np.int32), 16, _dev(G), 1)
    assert not empty.any()
    solver.close()


@pytest.mark.parametrize("n_frac", [0.25, 0.5, 0.8])
def test_find_mu_matches_oracle(gsk, n_frac):
    """mu for an electron count at several fillings; the search brackets by
    33-sections on the GPU, the oracle bisects: both reach the same root."""
    s, cols, eps, w, z, G, off = _case(64, 1.0, 1, 64)
    solver = gsk.from_system(s)
    sB = density.shift_traces(G, s.B, cols, off)
    kT = 0.3
    n_max = density.count_from_traces(sB, eps, w, 50.0, kT)
    n_elec = n_frac * n_max
    want = density.find_mu(sB, eps, w, kT, n_elec, -40.0, 40.0)
    mu, cnt = solver.find_mu(cols, eps, w, _dev(G), kT, n_elec, -40.0, 40.0)
    # |d mu| <= rounding of N / slope of N at the root
    h = 1e-4
    slope = (density.count_from_traces(sB, eps, w, want + h, kT)
             - density.count_from_traces(sB, eps, w, want - h, kT)) / (2 * h)
    assert slope > 0
    assert abs(mu - want) <= 1e-12 * n_max / slope + 1e-13
    assert abs(cnt - n_elec) <= 1e-11 * n_max
    solver.close()


def test_find_mu_unbracketed_is_einval(gsk):
    s, cols, eps, w, z, G, off = _case(64, 1.0, 1, 16)
    solver = gsk.from_system(s)
    with pytest.raises(gsk.GskError) as ei:
        solver.find_mu(cols, eps, w, _dev(G), 0.1, 1e9, -40.0, 40.0)
    assert ei.value.code == gsk.GSK_EINVAL
    solver.close()


def test_atom_pattern_matches_oracle(gsk):
    s = syn.make_system(300, 1.0 / 3.0, 2)
    solver = gsk.from_system(s)
    aptr, aidx = solver.atom_pattern()
    wptr, widx = density.atom_pattern(s.A, s.orb_offset, s.orb_count)
    assert np.array_equal(aptr, wptr) and np.array_equal(aidx, widx)
    solver.close()


@pytest.mark.parametrize("n_cols", [None, 53])
def test_icohp_matches_oracle(gsk, n_cols):
    """All columns (64 C atoms) and a subset of a C/H mix: C_IJ element by
    element; its sum against the energy trace."""
    if n_cols is None:
        s, cols, eps, w, z, G, off = _case(64, 1.0, 0, 16)
    else:
        s, cols, eps, w, z, G, off = _case(300, 1.0 / 3.0, 2, 16, n_cols=n_cols)
    rho = density.density_from_green(G, eps, w, -10.0, 0.1)
    aptr, aidx, want = density.icohp(rho, s.A, cols, off, s.orb_offset, s.orb_count)
    solver = gsk.from_system(s)
    C = torch.full((int(aptr[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    solver.icohp(cols, _dev(rho), C)
    torch.cuda.synchronize()
    got = C.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-13 * max(1.0, np.abs(want).max())
    assert np.isclose(got.sum(), solver.trace(cols, _dev(rho), 0), rtol=1e-12)
    solver.close()


def test_mu_from_traces_matches_find_mu(gsk):
    """gsk_mu_from_traces on the summed traces of two column halves (what the
    ranks of a sharded run exchange) gives the mu of gsk_find_mu on all columns."""
    from paper_1609_08377_gb300 import sharding

    s, cols, eps, w, z, G, off = _case(64, 1.0, 1, 64)
    solver = gsk.from_system(s)
    kT, n_elec = 0.3, 0.4 * density.count_from_traces(density.shift_traces(G, s.B, cols, off), eps, w, 50.0, 0.3)
    mu_all, cnt_all = solver.find_mu(cols, eps, w, _dev(G), kT, n_elec, -40.0, 40.0)
    halves = [sharding.shard_columns(cols, r, 2) for r in range(2)]
    s_sum = np.zeros(eps.size)
    for h in halves:
        Gh = dense.green_lu(s.A, s.B, z, h)
        s_sum += solver.shift_trace(h, eps.size, _dev(Gh), 1)
    mu, cnt = solver.mu_from_traces(eps, w, s_sum, kT, n_elec, -40.0, 40.0)
    assert abs(mu - mu_all) <= 1e-11 * max(1.0, abs(mu_all))
    assert abs(cnt - n_elec) <= 1e-11 * n_elec
    solver.close()
