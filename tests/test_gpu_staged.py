"""The staged SpMM of the FP32 inner CG, through the C ABI.

It computes the same product Y = B X as the per-atom gather kernel (the
inner CG's B-products of Sec. III-B's B^{-1} u), from a shared-memory copy of
each tile's neighbour rows, matrix values and indices. Checked:
  * against the FP64 product of the oracle's matrix B (row order of the
    library) on random FP32 lanes, to FP32 rounding, at 32, 64 and 128 lanes
    and on pencils whose tiles span one to hundreds of tiles, with a ragged
    last tile;
  * bitwise against the gather kernel at 32 lanes, where both sum every row
    in the same order;
  * inside gsk_solve: G against dense LU (O1) in both mixed modes at every
    lane width, the staged and gather runs agreeing to the mixed-mode bar,
    and bitwise repeatability (graph and host loop).
"""

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


@pytest.fixture(scope="module")
def systems():
    return {"c64": syn.make_system(64, 1.0, 0), "ch1k": syn.make_system(1000, 1.0 / 3.0, 0),
            "ch20k": syn.make_system(20000, 1.0 / 3.0, 0)}


def _lib_order_B(solver, s):
    """B with rows and columns in the library's order (FP64)."""
    perm = solver.row_order()                 # caller row i -> library row perm[i]
    P = sp.csr_matrix((np.ones(s.M), (perm, np.arange(s.M))), shape=(s.M, s.M))
    return (P @ s.B @ P.T).tocsr()


@pytest.mark.parametrize("name", ["c64", "ch1k", "ch20k"])
@pytest.mark.parametrize("W", [32, 64, 128])
def test_staged_product_matches_fp64(gsk, systems, name, W):
    s = systems[name]
    solver = gsk.from_system(s)
    Bl = _lib_order_B(solver, s)
    rng = np.random.default_rng(W)
    X = rng.standard_normal((s.M, W)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    ref = Bl @ X.astype(np.float64)
    # FP32 products with FP32-rounded values: |error| <= ~(nnz per row) * 2^-24 * sum |B_ik X_k|
    bound = (abs(Bl) @ np.abs(X.astype(np.float64))) * 3e-6
    out = {}
    for which in (1, 2):
        Yd = torch.full((s.M, W), np.nan, dtype=torch.float32, device="cuda")
        solver.spmm(which, gsk.GSK_MIXED, W, Xd, Yd)
        torch.cuda.synchronize()
        out[which] = Yd.cpu().numpy()
        assert np.isfinite(out[which]).all(), which
        assert (np.abs(out[which] - ref) <= bound + 1e-30).all(), which
    # the staged kernel sums each row like the 32-lane gather, at every width
    Yg32 = torch.empty((s.M, 32), dtype=torch.float32, device="cuda")
    for q in range(W // 32):
        solver.spmm(1, gsk.GSK_MIXED, 32, Xd[:, 32 * q:32 * (q + 1)].contiguous(), Yg32)
        torch.cuda.synchronize()
        assert np.array_equal(out[2][:, 32 * q:32 * (q + 1)], Yg32.cpu().numpy())
    solver.close()


def _solve(gsk, solver, z, cols, **kw):
    off = solver.pattern_offsets(cols)
    G = torch.zeros(int(off[-1]) * len(z), dtype=torch.complex128, device="cuda")
    it, st, rs = solver.solve(z, cols, G, **kw)
    torch.cuda.synchronize()
    return G.cpu().numpy().reshape(int(off[-1]), len(z)), it, st


@pytest.mark.parametrize("kern", ["staged"])
@pytest.mark.parametrize("prec", ["mixed", "mixed_df"])
@pytest.mark.parametrize("W", [32, 64, 128])
def test_solve_staged_matches_lu(gsk, systems, kern, prec, W):
    s = systems["c64"]
    z = syn.shifts(syn.energy_grid(16), 0.1)
    cols = np.arange(0, s.M, 3, dtype=np.int32)
    R = dense.green_lu(s.A, s.B, z, cols)
    solver = gsk.from_system(s)
    Gt, it_t, st_t = _solve(gsk, solver, z, cols, precision=prec, tol=1e-10, batch_w=W, spmm_kernel=kern)
    assert solver.last_stats()["spmm_kernel"] == gsk.GSK_SPMM_STAGED
    Gg, it_g, st_g = _solve(gsk, solver, z, cols, precision=prec, tol=1e-10, batch_w=W, spmm_kernel="gather")
    assert solver.last_stats()["spmm_kernel"] == gsk.GSK_SPMM_GATHER
    assert (st_t == gsk.GSK_CONVERGED).all() and (st_g == gsk.GSK_CONVERGED).all()
    scale = np.abs(R).max()
    assert np.abs(Gt - R).max() / scale <= 1e-8
    assert np.abs(Gt - Gg).max() / scale <= 1e-8
    # beyond M Lanczos steps (M = 256 here, about 1,500 steps taken) the
    # iterates depend on rounding order, so the two kernels' step counts agree
    # only roughly while G agrees to the bar
    assert np.abs(it_t.astype(int) - it_g).max() <= 0.1 * it_g.max() + 10
    solver.close()


def test_default_kernel_by_lane_width(gsk, systems):
    """Without an autotuner pick, the mixed modes run the staged product at 32
    lanes and the gather product at 64 and 128 (the measured rule)."""
    s = systems["ch1k"]
    solver = gsk.from_system(s)
    z = syn.energy_grid(8).astype(np.complex128) + 1j
    cols = np.arange(4, dtype=np.int32)
    for W, kind in ((32, gsk.GSK_SPMM_STAGED), (64, gsk.GSK_SPMM_GATHER), (128, gsk.GSK_SPMM_GATHER)):
        _solve(gsk, solver, z, cols, eta=np.full(cols.size, 0.2), precision="mixed_df", tol=1e-8, batch_w=W)
        assert solver.last_stats()["spmm_kernel"] == kind, W
    solver.close()


def test_solve_staged_ch1k_per_column_eta(gsk, systems):
    s = systems["ch1k"]
    eps = syn.energy_grid(32)
    cols = syn.column_subset(s.M, 96, 5).astype(np.int32)
    eta = syn.eta_per_column(cols.size, 5)
    solver = gsk.from_system(s)
    z = eps.astype(np.complex128) + 1j
    G, it, st = _solve(gsk, solver, z, cols, eta=eta, precision="mixed_df", tol=1e-10, batch_w=64,
                       spmm_kernel="staged")
    assert solver.last_stats()["spmm_kernel"] == gsk.GSK_SPMM_STAGED
    assert (st == gsk.GSK_CONVERGED).all()
    off = solver.pattern_offsets(cols)
    worst = 0.0
    for c in range(0, cols.size, 7):
        R = dense.green_lu(s.A, s.B, syn.shifts(eps, float(eta[c])), cols[c:c + 1])
        worst = max(worst, float(np.abs(G[off[c]:off[c + 1]] - R).max() / np.abs(R).max()))
    assert worst <= 1e-8, worst
    solver.close()


@pytest.mark.parametrize("kern", ["staged", "gather"])
def test_staged_bitwise_repeatable(gsk, systems, kern):
    s = systems["c64"]
    z = syn.shifts(syn.energy_grid(16), 0.1)
    cols = np.arange(0, s.M, 2, dtype=np.int32)
    solver = gsk.from_system(s)
    Ga, ia, _ = _solve(gsk, solver, z, cols, precision="mixed", tol=1e-10, batch_w=64, spmm_kernel=kern)
    Gb, ib, _ = _solve(gsk, solver, z, cols, precision="mixed", tol=1e-10, batch_w=64, spmm_kernel=kern)
    Gc, ic, _ = _solve(gsk, solver, z, cols, precision="mixed", tol=1e-10, batch_w=64, spmm_kernel=kern,
                       use_graph=0)
    assert np.array_equal(Ga, Gb) and np.array_equal(ia, ib)
    assert np.array_equal(Ga, Gc) and np.array_equal(ia, ic)
    solver.close()


def test_staged_refuses_fp64(gsk, systems):
    s = systems["c64"]
    solver = gsk.from_system(s)
    z = syn.shifts(syn.energy_grid(4), 0.1)
    cols = np.arange(4, dtype=np.int32)
    off = solver.pattern_offsets(cols)
    G = torch.zeros(int(off[-1]) * 4, dtype=torch.complex128, device="cuda")
    for kern in ("staged",):
        with pytest.raises(gsk.GskError) as e:
            solver.solve(z, cols, G, precision="fp64", spmm_kernel=kern)
        assert e.value.code == gsk.GSK_ENOTSUP
    X = torch.zeros((s.M, 32), dtype=torch.float64, device="cuda")
    for which in (2,):
        with pytest.raises(gsk.GskError) as e:
            solver.spmm(which, gsk.GSK_FP64, 32, X, X)
        assert e.value.code == gsk.GSK_ENOTSUP
    solver.close()
