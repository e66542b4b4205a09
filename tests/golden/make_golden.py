"""Write oracle reference values for sampled columns of the large workloads.

Calls only the CPU oracle (oracle/krylov.py: the naive FP64 B-Lanczos of
Sec. III-B, one column at a time or a batch of columns through the oracle's
C loops) and the seeded input generator. For each sampled column of a
workload it stores: the column, its damping eta, the oracle's step count at
the 1e-8 residual level, and G on the column's pattern at every
shift_stride-th shift, from a run to a 1e-10 residual. Usage:

    python tests/golden/make_golden.py ch20k 0 3            # workload, first, count (one column at a time)
    python tests/golden/make_golden.py ch100k --batch 0.2:24 0.1:24
        # a batch: the first 24 columns of the seeded subset with eta = 0.2
        # and the first 24 with eta = 0.1 that have no stored file yet
    python tests/golden/make_golden.py ch1m --steps 16 16
        # the first 16 columns of the seeded subset, stopped after exactly 16
        # Lanczos steps (files <workload>_steps<n>_col<j>.json)

The --steps mode is for pencils where a converged oracle column takes hours:
after n steps both the oracle and the solver return the Galerkin solution of
the n-step Krylov subspace, x_n(z) = Q_n (z - T_n)^{-1} beta_0 e_1 (Sec.
III-B). The file also stores, per column, how far that G moves when the
oracle's inner CG stops at a relative residual of 1e-10 instead of 1e-14
("spread_bsolve_1e-10"): the rounding sensitivity of the unconverged
iterate, measured, from which a test sets its tolerance.

Columns are taken in the order of the workload's seeded column subset
(synthetic.column_subset), each with its seeded damping
(synthetic.eta_per_column).
"""

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import krylov  # noqa: E402
from paper_1609_08377_gb300 import synthetic as syn  # noqa: E402

SHIFT_STRIDE = 8
HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE_ONE = ("oracle/krylov.py lanczos_column (naive FP64 B-Lanczos, CG inner solves to 1e-14), "
              "tol 1e-10; Sec. III-B of arXiv:1609.08377 (generalized shifted equations)")
SOURCE_STEPS = ("oracle/krylov.py lanczos_batch (naive FP64 B-Lanczos over a batch of columns, C loops in "
                "oracle/o3_batch.c, CG inner solves to 1e-14) stopped after a fixed number of steps n: "
                "G_n = Q_n (z - T_n)^-1 beta_0 e_1; Sec. III-B of arXiv:1609.08377")
SOURCE_BATCH = ("oracle/krylov.py lanczos_batch (naive FP64 B-Lanczos over a batch of columns, C loops in "
                "oracle/o3_batch.c, CG inner solves to 1e-14), tol 1e-10; Sec. III-B of arXiv:1609.08377 "
                "(generalized shifted equations)")


def sample(name: str, seed: int = 0):
    """Columns of the workload's seeded subset, one per damping class first."""
    wl = syn.WORKLOADS[name]
    s = syn.make_system(wl.n_atoms, wl.c_fraction, seed)
    n_cols = wl.n_cols if wl.n_cols is not None else s.M
    cols = syn.column_subset(s.M, n_cols, seed)
    eta = syn.eta_per_column(cols.size, seed) if wl.eta is None else np.full(cols.size, wl.eta)
    order = []
    for e in (0.05, 0.1, 0.2):
        idx = np.nonzero(np.isclose(eta, e))[0]
        order.extend(idx[:2].tolist())
    return wl, s, cols, eta, order


def _path(name, j):
    return os.path.join(HERE, f"{name}_col{j}.json")


def _record(name, wl, j, e, r, seconds, source):
    return {
        "source": source, "workload": name, "seed": 0, "column": int(j), "eta": float(e),
        "n_shifts": int(wl.n_shifts), "shift_stride": SHIFT_STRIDE,
        "iters_1e-8": int(r.reached.get(1e-8, -1)), "iters_1e-10": int(r.iters),
        "converged": bool(r.converged), "seconds": seconds,
        "G_re": [[float(v) for v in row] for row in r.G[:, ::SHIFT_STRIDE].real],
        "G_im": [[float(v) for v in row] for row in r.G[:, ::SHIFT_STRIDE].imag],
    }


def one_by_one(name, first, count):
    wl, s, cols, eta, order = sample(name)
    eps = syn.energy_grid(wl.n_shifts)
    for t in order[first:first + count]:
        j, e = int(cols[t]), float(eta[t])
        t0 = time.time()
        r = krylov.lanczos_column(s.A, s.B, j, syn.shifts(eps, e), tol=1e-10, max_iter=60000,
                                  milestones=(1e-8,))
        out = _record(name, wl, j, e, r, time.time() - t0, SOURCE_ONE)
        with open(_path(name, j), "w") as f:
            json.dump(out, f)
        print(name, j, e, out["iters_1e-8"], out["iters_1e-10"], round(out["seconds"]), flush=True)


def batch(name, classes):
    """classes: list of (eta, count); one oracle batch over all chosen columns."""
    wl = syn.WORKLOADS[name]
    s = syn.make_system(wl.n_atoms, wl.c_fraction, 0)
    n_cols = wl.n_cols if wl.n_cols is not None else s.M
    cols = syn.column_subset(s.M, n_cols, 0)
    eta = syn.eta_per_column(cols.size, 0) if wl.eta is None else np.full(cols.size, wl.eta)
    pick = []
    for e, k in classes:
        got = 0
        for t in np.nonzero(np.isclose(eta, e))[0].tolist():
            if got == k:
                break
            if os.path.exists(_path(name, int(cols[t]))):
                continue
            pick.append(t)
            got += 1
    js = [int(cols[t]) for t in pick]
    es = [float(eta[t]) for t in pick]
    eps = syn.energy_grid(wl.n_shifts)
    print(name, "batch of", len(js), "columns:", list(zip(js, es)), "threads", krylov.set_threads(0), flush=True)
    t0 = time.time()

    def progress(n, n_act):
        if n % 500 == 0:
            print(f"step {n}: {n_act} columns active, {time.time() - t0:.0f} s", flush=True)

    def done(c, r):
        out = _record(name, wl, js[c], es[c], r, time.time() - t0, SOURCE_BATCH)
        with open(_path(name, js[c]), "w") as f:
            json.dump(out, f)
        print(name, js[c], es[c], out["iters_1e-8"], out["iters_1e-10"], round(out["seconds"]), flush=True)

    krylov.lanczos_batch(s.A, s.B, js, [syn.shifts(eps, e) for e in es], tol=1e-10, max_iter=60000,
                         milestones=(1e-8,), progress=progress, on_done=done)


def fixed_steps(name, n, k):
    """The first k columns of the seeded subset after exactly n oracle steps."""
    wl = syn.WORKLOADS[name]
    t0 = time.time()
    s = syn.make_system(wl.n_atoms, wl.c_fraction, 0)
    n_cols = wl.n_cols if wl.n_cols is not None else s.M
    cols = syn.column_subset(s.M, n_cols, 0)
    eta = syn.eta_per_column(cols.size, 0) if wl.eta is None else np.full(cols.size, wl.eta)
    js = [int(j) for j in cols[:k]]
    es = [float(e) for e in eta[:k]]
    eps = syn.energy_grid(wl.n_shifts)
    z = [syn.shifts(eps, e) for e in es]
    print(name, "pencil", s.M, "rows", s.A.nnz, "nnz", f"{time.time() - t0:.0f} s; columns", list(zip(js, es)),
          "threads", krylov.set_threads(0), flush=True)

    def run(btol):
        t1 = time.time()
        r = krylov.lanczos_batch(s.A, s.B, js, z, tol=0.0, max_iter=n, check_every=n, bsolve_tol=btol)
        print(f"{n} steps, inner CG to {btol:g}: {time.time() - t1:.0f} s", flush=True)
        return r, time.time() - t1

    ref, sec = run(1e-14)
    loose, _ = run(1e-10)
    for c, j in enumerate(js):
        R = ref[c].G[:, ::SHIFT_STRIDE]
        L = loose[c].G[:, ::SHIFT_STRIDE]
        spread = float(np.abs(R - L).max() / np.abs(R).max())
        out = {
            "source": SOURCE_STEPS, "workload": name, "seed": 0, "column": j, "eta": es[c],
            "n_shifts": int(wl.n_shifts), "shift_stride": SHIFT_STRIDE, "steps": int(n),
            "spread_bsolve_1e-10": spread, "seconds": sec,
            "G_re": [[float(v) for v in row] for row in R.real],
            "G_im": [[float(v) for v in row] for row in R.imag],
        }
        with open(os.path.join(HERE, f"{name}_steps{n}_col{j}.json"), "w") as f:
            json.dump(out, f)
        print(name, j, es[c], "spread", f"{spread:.2e}", flush=True)


def main():
    name = sys.argv[1]
    if sys.argv[2] == "--steps":
        fixed_steps(name, int(sys.argv[3]), int(sys.argv[4]))
    elif sys.argv[2] == "--batch":
        classes = [(float(a), int(b)) for a, b in (x.split(":") for x in sys.argv[3:])]
        batch(name, classes)
    else:
        one_by_one(name, int(sys.argv[2]), int(sys.argv[3]))


if __name__ == "__main__":
    main()
