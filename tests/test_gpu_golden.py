"""Full-size parity: sampled columns of the 20,000-, 100,000- and
1,000,000-atom workloads against stored oracle references.

The stored references (tests/golden/*.json) were written by
tests/golden/make_golden.py, which calls only the CPU oracle (the naive FP64
B-Lanczos of Sec. III-B, one column at a time or a batch of columns, run to a
1e-10 residual). The solver runs in the workload's configuration (128 or 64
shifts, per-column damping, tol 1e-8) in the double-float mixed mode at the
lane widths the benchmark uses, and in plain FP64 on a subset, and must meet
|Delta G| / max |G| <= 1e-8 on every stored shift of every stored column; its
step count must agree with the oracle's step count at the 1e-8 level (the
oracle checks the residual every 10 steps). At 10^6 atoms G_ij from column j
also equals G_ji from column i for a neighbour pair (G(z)^T = G(z) for
symmetric A and B), the property checked where no stored columns exist.
Where a converged oracle column is out of reach (10^6 atoms), stored oracle
columns after a fixed number n of Lanczos steps are compared with the
solver stopped after the same n steps (tests/golden/*_steps*_col*.json).
"""

import glob
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1609_08377_gb300 import synthetic as syn  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
_SYSTEMS = {}


def _golden(name):
    return [json.load(open(p)) for p in sorted(glob.glob(os.path.join(HERE, "golden", f"{name}_col*.json")))]


def _system(name):
    if name not in _SYSTEMS:
        _SYSTEMS.clear()                          # keep one large pencil in memory at a time
        wl = syn.WORKLOADS[name]
        _SYSTEMS[name] = syn.make_system(wl.n_atoms, wl.c_fraction, 0)
    return _SYSTEMS[name]


def _check(name, prec, W, pick=None, extra_cols=()):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    refs = _golden(name)
    if not refs:
        pytest.skip(f"no stored oracle columns for {name}")
    if pick is not None:
        refs = pick(refs)
    from paper_1609_08377_gb300 import gsk

    wl = syn.WORKLOADS[name]
    s = _system(name)
    solver = gsk.from_system(s)
    cols = np.array([r["column"] for r in refs] + list(extra_cols), dtype=np.int32)
    eta = np.array([r["eta"] for r in refs] + [refs[0]["eta"]] * len(extra_cols))
    eps = syn.energy_grid(wl.n_shifts)
    z = eps.astype(np.complex128) + 1j
    off = solver.pattern_offsets(cols)
    G = torch.zeros(int(off[-1]) * wl.n_shifts, dtype=torch.complex128, device="cuda")
    it, st, _ = solver.solve(z, cols, G, eta=eta, precision=prec, tol=1e-8, batch_w=W, sched="fifo")
    torch.cuda.synchronize()
    Gh = G.cpu().numpy().reshape(int(off[-1]), wl.n_shifts)
    assert (st == gsk.GSK_CONVERGED).all()
    worst = 0.0
    for c, r in enumerate(refs):
        R = np.array(r["G_re"]) + 1j * np.array(r["G_im"])
        got = Gh[off[c]:off[c + 1], ::r["shift_stride"]]
        err = np.abs(got - R).max() / np.abs(R).max()
        worst = max(worst, err)
        assert err <= 1e-8, (r["column"], err)
        n_or = r["iters_1e-8"]
        # an inexact inner solve (FP32 passes to 3e-6 in the mixed modes) delays
        # convergence by about 1-2 %; the FP64 inner solve (1e-12) tracks the oracle
        slack = 0.02 if prec == "fp64" else 0.04
        assert abs(it[c] - n_or) <= slack * n_or + 10, (r["column"], it[c], n_or)
    return solver, s, cols, off, Gh, worst


@pytest.mark.parametrize("name,prec,W", [("ch20k", "mixed_df", 32), ("ch100k", "mixed_df", 32),
                                         ("ch100k", "mixed_df", 64), ("ch100k", "mixed_df", 128)])
def test_golden_columns(name, prec, W):
    """At 32 lanes the mixed modes run the staged inner-CG product (the
    benchmark's configuration), at 64 and 128 the gather product."""
    solver, *_ = _check(name, prec, W)
    assert solver.last_stats()["spmm_kernel"] == (2 if W == 32 else 1)
    solver.close()


@pytest.mark.parametrize("name,n", [("ch20k", 2), ("ch100k", 8)])
def test_golden_columns_plain_fp64(name, n):
    """Plain FP64 on the stored columns that converge soonest (eta = 0.2)."""
    solver, *_ = _check(name, "fp64", 32, pick=lambda refs: sorted(refs, key=lambda r: r["iters_1e-8"])[:n])
    solver.close()


def test_1m_symmetry_and_stored_columns():
    """The 1,000,000-atom pencil (M ~ 2e6), where the oracle takes hours per
    column: G_ij(z) from column j equals G_ji(z) from column i for a
    neighbour pair (a property that holds at any size), and the stored oracle
    columns of this workload, if any, to 1e-8."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_08377_gb300 import gsk

    refs = _golden("ch1m")
    wl = syn.WORKLOADS["ch1m"]
    s = _system("ch1m")
    A = s.A
    if refs:
        j = int(refs[0]["column"])
        eta_j = float(refs[0]["eta"])
    else:
        cols_all = syn.column_subset(s.M, wl.n_cols, 0)
        eta_all = syn.eta_per_column(cols_all.size, 0)
        t = int(np.nonzero(np.isclose(eta_all, 0.2))[0][0])
        j, eta_j = int(cols_all[t]), 0.2
    nb = A.indices[A.indptr[j]:A.indptr[j + 1]]
    others = set(int(r["column"]) for r in refs)
    i = int(next(x for x in nb[::-1] if x != j and int(x) not in others))
    solver = gsk.from_system(s)
    cols = np.array([int(r["column"]) for r in refs] + ([] if refs else [j]) + [i], dtype=np.int32)
    eta = np.array([float(r["eta"]) for r in refs] + ([] if refs else [eta_j]) + [eta_j])
    eps = syn.energy_grid(wl.n_shifts)
    z = eps.astype(np.complex128) + 1j
    off = solver.pattern_offsets(cols)
    G = torch.zeros(int(off[-1]) * wl.n_shifts, dtype=torch.complex128, device="cuda")
    it, st, _ = solver.solve(z, cols, G, eta=eta, precision="mixed_df", tol=1e-8, batch_w=32, sched="fifo")
    torch.cuda.synchronize()
    assert (st == gsk.GSK_CONVERGED).all()
    Gh = G.cpu().numpy().reshape(int(off[-1]), wl.n_shifts)
    for c, r in enumerate(refs):
        R = np.array(r["G_re"]) + 1j * np.array(r["G_im"])
        got = Gh[off[c]:off[c + 1], ::r["shift_stride"]]
        assert np.abs(got - R).max() / np.abs(R).max() <= 1e-8, r["column"]
    c_j = int(np.nonzero(cols == j)[0][0])
    c_i = int(np.nonzero(cols == i)[0][0])
    rows_j = A.indices[A.indptr[j]:A.indptr[j + 1]]
    rows_i = A.indices[A.indptr[i]:A.indptr[i + 1]]
    g_ij = Gh[off[c_j] + int(np.nonzero(rows_j == i)[0][0])]     # row i of column j
    g_ji = Gh[off[c_i] + int(np.nonzero(rows_i == j)[0][0])]     # row j of column i
    assert np.abs(g_ij - g_ji).max() <= 1e-8 * np.abs(Gh).max()
    solver.close()


def _steps_golden(name):
    return [json.load(open(p))
            for p in sorted(glob.glob(os.path.join(HERE, "golden", f"{name}_steps*_col*.json")))]


@pytest.mark.parametrize("prec", ["fp64", "mixed_df"])
def test_1m_fixed_steps_against_oracle(prec):
    """The 1,000,000-atom pencil against the oracle where a converged oracle
    column is out of reach: after exactly n Lanczos steps both sides return
    the Galerkin solution of the n-step Krylov subspace, x_n(z) = Q_n (z -
    T_n)^{-1} beta_0 e_1 (Sec. III-B), on 16 seeded columns of all three
    damping classes. An unconverged iterate carries the rounding of the inner
    B-solves, amplified near the early Ritz values: each stored column gives
    how far the oracle's own G_n moves when its inner CG stops at 1e-10
    instead of 1e-14 (the spread; 9e-10 to 2.4e-4 over these columns, largest
    at eta = 0.05). The change is first order in the inner-solve error, so the
    FP64 solve (inner CG to 1e-14, 1e-4 of the probe's error) must agree to
    1e-3 of the spread (at least 1e-10), and the double-float mode (an FP32
    pass to 3e-6 and one refinement pass, about 1e-11) to twice the spread
    (at least 1e-9). This checks the solver at 10^6 atoms against the oracle;
    the converged 1e-8 check of the smaller workloads is not reachable here."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    refs = _steps_golden("ch1m")
    if not refs:
        pytest.skip("no stored fixed-step oracle columns for ch1m")
    from paper_1609_08377_gb300 import gsk

    n = int(refs[0]["steps"])
    assert all(int(r["steps"]) == n for r in refs)
    wl = syn.WORKLOADS["ch1m"]
    s = _system("ch1m")
    solver = gsk.from_system(s)
    cols = np.array([int(r["column"]) for r in refs], dtype=np.int32)
    eta = np.array([float(r["eta"]) for r in refs])
    eps = syn.energy_grid(wl.n_shifts)
    z = eps.astype(np.complex128) + 1j
    off = solver.pattern_offsets(cols)
    G = torch.zeros(int(off[-1]) * wl.n_shifts, dtype=torch.complex128, device="cuda")
    kw = dict(inner_tol=1e-14) if prec == "fp64" else {}
    it, st, _ = solver.solve(z, cols, G, eta=eta, precision=prec, tol=1e-30, max_iter=n, batch_w=32,
                             sched="fifo", **kw)
    torch.cuda.synchronize()
    assert (it == n).all() and (st == gsk.GSK_NOT_CONVERGED).all()
    Gh = G.cpu().numpy().reshape(int(off[-1]), wl.n_shifts)
    errs = []
    for c, r in enumerate(refs):
        R = np.array(r["G_re"]) + 1j * np.array(r["G_im"])
        got = Gh[off[c]:off[c + 1], ::r["shift_stride"]]
        err = np.abs(got - R).max() / np.abs(R).max()
        spread = float(r["spread_bsolve_1e-10"])
        bar = max(1e-10, 1e-3 * spread) if prec == "fp64" else max(1e-9, 2.0 * spread)
        errs.append((r["column"], err, bar))
        assert err <= bar, (r["column"], err, bar)
    print(prec, "worst |dG|/max|G| after", n, "steps:", max(e for _, e, _ in errs))
    solver.close()
