"""Real-space projection on the GPU (gsk_marnoldi_projected) against the
oracle (Sec. III-B): region sizes exactly, rho on the full pattern within
the multiple Arnoldi tolerances (see tests/test_gpu_marnoldi.py) computed on
each column's projected pencil, and the whole-system region against the
unprojected GPU path."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import marnoldi as ma, projection as pj  # noqa: E402
from paper_1609_08377_gb300 import synthetic as syn  # noqa: E402

U = 2.0 ** -53


@pytest.fixture(scope="module")
def gsk():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_08377_gb300 import gsk as g
    return g


@pytest.fixture(scope="module")
def ch1k():
    return syn.make_system(1000, 1.0 / 3.0, 0)


def _box(s):
    return (s.box,) * 3 if np.isscalar(s.box) else tuple(s.box)


def _rho(solver, cols):
    off = solver.pattern_offsets(cols)
    return off, torch.full((int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("kappa,nu,n_cols", [(100, 30, 45), (40, 20, 9)])
def test_projected_matches_oracle(gsk, ch1k, kappa, nu, n_cols):
    s = ch1k
    box = _box(s)
    cols = syn.column_subset(s.M, n_cols, 4)
    solver = gsk.from_system(s)
    off, rho = _rho(solver, cols)
    ritz, weight, charge, rank, m_local = solver.marnoldi_projected(cols, kappa, nu, -10.0, 0.1, rho, box=box)
    torch.cuda.synchronize()
    got = rho.cpu().numpy()
    atom_of = s.atom_of_row()
    checked = 0
    for c, j in enumerate(cols.tolist()):
        o = pj.projected_marnoldi_column(s.A, s.B, s.orb_offset, s.orb_count, s.pos, box, j, kappa, nu,
                                         mu=-10.0, kT=0.1)
        assert m_local[c] == o["M_local"]
        assert abs(charge[c, :rank[c]].sum() - 1.0) < 1e-10
        atoms = pj.region_atoms(s.pos, int(atom_of[j]), kappa, box)
        Ap, Bp, rows = pj.projected_pencil(s.A, s.B, s.orb_offset, s.orb_count, atoms)
        jl = int(np.nonzero(rows == j)[0][0])
        sines = ma.principal_sines(Ap, Bp, jl, nu)
        if np.any(np.abs(sines / ma.RANK_TOL - 1.0) < 0.1):
            continue
        kept = sines[sines >= ma.RANK_TOL]
        sig = kept.min() if kept.size else 1.0
        p = ma.marnoldi_column(Ap, Bp, jl, nu, mu=-10.0, kT=0.1, seed_tol=1e-13)
        q = ma.marnoldi_column(Ap, Bp, jl, nu, mu=-10.0, kT=0.1)
        k_rho = np.abs(p["rho"] - q["rho"]).max() / np.abs(q["rho"]).max() / 1e-13 if p["eps"].size == q["eps"].size else 0.0
        assert rank[c] == o["eps"].size
        tol = (3e-11 + 20 * U / sig + 1e-14 * k_rho) * np.abs(o["rho"]).max()
        err = np.abs(got[off[c]:off[c + 1]] - o["rho"]).max()
        assert err <= tol, (j, err, tol)
        checked += 1
    assert checked >= n_cols - 2
    solver.close()


def test_whole_system_region_equals_unprojected(gsk):
    """kappa >= number of atoms: every region is the whole pencil, so the
    projected path reproduces gsk_marnoldi column for column, up to the
    rounding of a different row order (the projected pencils carry no
    positions, so their rows are not reordered along a space-filling curve):
    the 3e-11 floor of the multiple Arnoldi comparisons."""
    s = syn.make_system(64, 1.0, 0)
    cols = np.array([0, 9, 100, 255], dtype=np.int32)
    solver = gsk.from_system(s)
    off, rho_p = _rho(solver, cols)
    _, rho_u = _rho(solver, cols)
    rp, wp, qp, kp, ml = solver.marnoldi_projected(cols, 64, 20, -10.0, 0.1, rho_p, box=_box(s))
    ru, wu, qu, ku = solver.marnoldi(cols, 20, -10.0, 0.1, rho_u)
    torch.cuda.synchronize()
    assert (ml == s.M).all() and (kp == ku).all()
    a, b = rho_p.cpu().numpy(), rho_u.cpu().numpy()
    assert np.abs(a - b).max() <= 3e-11 * np.abs(b).max()
    solver.close()


def test_projection_needs_positions(gsk):
    s = syn.make_system(64, 1.0, 0)
    solver = gsk.from_system(s, pos=False)
    _, rho = _rho(solver, np.array([0], np.int32))
    with pytest.raises(gsk.GskError) as ei:
        solver.marnoldi_projected(np.array([0], np.int32), 10, 20, -10.0, 0.1, rho)
    assert ei.value.code == gsk.GSK_EINVAL
    solver.close()
