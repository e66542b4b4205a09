"""Pins of the real-space projection oracle (Sec. III-B): the region rule
against brute force, exactness when the region is everything or a
decoupled cluster, the minimum-image convention, and that a region wider
than the cutoff keeps all of P(j)."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import marnoldi as ma, projection as pj
from paper_1609_08377_gb300 import synthetic as syn


@pytest.fixture(scope="module")
def ch1k():
    return syn.make_system(1000, 1.0 / 3.0, 0)


def test_region_rule_bruteforce(ch1k):
    """kappa or more atoms, and every atom closer than any excluded one."""
    s = ch1k
    box = (s.box,) * 3 if np.isscalar(s.box) else s.box
    for J, kappa in ((0, 100), (17, 37), (999, 1)):
        atoms = pj.region_atoms(s.pos, J, kappa, box)
        assert atoms.size >= kappa and J in atoms
        d = np.array([min(np.linalg.norm(s.pos[a] - s.pos[J] - np.array(box) * k)
                          for k in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1])).T.reshape(-1, 3))
                      for a in range(s.n_atoms)])
        inside = np.zeros(s.n_atoms, bool)
        inside[atoms] = True
        assert d[inside].max() <= d[~inside].min() + 1e-12
        assert (np.sort(d)[kappa - 1] >= d[inside]).all()


def test_minimum_image():
    pos = np.array([[0.1, 5.0, 5.0], [9.9, 5.0, 5.0], [5.0, 5.0, 5.0]])
    d2 = pj.min_image_dist2(pos, 0, (10.0, 10.0, 10.0))
    assert np.isclose(d2[1], 0.04) and np.isclose(d2[2], 24.01)
    assert list(pj.region_atoms(pos, 0, 2, (10.0, 10.0, 10.0))) == [0, 1]
    assert list(pj.region_atoms(pos, 0, 2, None)) == [0, 2]


def test_whole_system_region_is_unprojected(ch1k):
    s = ch1k
    box = (s.box,) * 3 if np.isscalar(s.box) else s.box
    for j in (0, 5, 1234):
        o = pj.projected_marnoldi_column(s.A, s.B, s.orb_offset, s.orb_count, s.pos, box, j, s.n_atoms, 20,
                                         mu=-10.0, kT=0.1)
        ref = ma.marnoldi_column(s.A, s.B, j, 20, mu=-10.0, kT=0.1)
        assert o["M_local"] == s.M
        assert np.abs(o["rho"] - ref["rho"]).max() <= 1e-12 * np.abs(ref["rho"]).max()
        assert np.allclose(o["eps"], ref["eps"], atol=1e-10)


def test_decoupled_cluster_is_exact():
    """Two copies of a 64-atom pencil placed far apart (block-diagonal A, B):
    with kappa = 64 the region is the column's own copy, which is decoupled,
    so the projected answer equals the unprojected one."""
    s = syn.make_system(64, 1.0, 0)
    A = sp.block_diag([s.A, s.A], format="csr")
    B = sp.block_diag([s.B, s.B], format="csr")
    pos = np.vstack([s.pos, s.pos + 1000.0])
    off = np.concatenate([s.orb_offset, s.orb_offset + s.M])
    cnt = np.concatenate([s.orb_count, s.orb_count])
    for j in (3, s.M + 77):
        o = pj.projected_marnoldi_column(A, B, off, cnt, pos, None, j, 64, 20, mu=-10.0, kT=0.1)
        ref = ma.marnoldi_column(A, B, j, 20, mu=-10.0, kT=0.1)
        assert o["M_local"] == s.M
        assert np.abs(o["rho"] - ref["rho"]).max() <= 1e-12 * np.abs(ref["rho"]).max()


def test_region_wider_than_cutoff_keeps_pattern(ch1k):
    """kappa = 100 atoms at 0.1 atoms/A^3 reach about 6.2 A, beyond the 5 A
    cutoff, so every row of P(j) is inside and rho has no forced zeros; the
    projected problem has M' in the paper's 200-400 range."""
    s = ch1k
    box = (s.box,) * 3 if np.isscalar(s.box) else s.box
    for j in (0, 700, 1500):
        o = pj.projected_marnoldi_column(s.A, s.B, s.orb_offset, s.orb_count, s.pos, box, j, 100, 30,
                                         mu=-10.0, kT=0.1)
        assert (o["rho"] != 0.0).all()
        assert 150 <= o["M_local"] <= 400, o["M_local"]
        assert abs(o["q"].sum() - 1.0) < 1e-6
