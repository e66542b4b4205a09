"""Write oracle reference values for sampled columns of the large workloads.

Calls only the CPU oracle (oracle/krylov.py, the naive FP64 B-Lanczos of
Sec. III-B) and the seeded input generator. For each sampled column of a
workload it stores: the column, its damping eta, the oracle's step count at
the 1e-8 residual level, and G on the column's pattern at every shift_stride-th
shift, from a run to a 1e-10 residual. Usage:

    python tests/golden/make_golden.py ch20k 0 3      # workload, first, count
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


def main():
    name, first, count = sys.argv[1], int(sys.argv[2]), int(sys.argv[3])
    wl, s, cols, eta, order = sample(name)
    eps = syn.energy_grid(wl.n_shifts)
    for t in order[first:first + count]:
        j, e = int(cols[t]), float(eta[t])
        t0 = time.time()
        r = krylov.lanczos_column(s.A, s.B, j, syn.shifts(eps, e), tol=1e-10, max_iter=60000,
                                  milestones=(1e-8,))
        out = {
            "source": "oracle/krylov.py lanczos_column (naive FP64 B-Lanczos, CG inner solves to 1e-14), "
                      "tol 1e-10; Sec. III-B of arXiv:1609.08377 (generalized shifted equations)",
            "workload": name, "seed": 0, "column": j, "eta": e, "n_shifts": int(wl.n_shifts),
            "shift_stride": SHIFT_STRIDE, "iters_1e-8": int(r.reached.get(1e-8, -1)),
            "iters_1e-10": int(r.iters), "converged": bool(r.converged), "seconds": time.time() - t0,
            "G_re": [[float(v) for v in row] for row in r.G[:, ::SHIFT_STRIDE].real],
            "G_im": [[float(v) for v in row] for row in r.G[:, ::SHIFT_STRIDE].imag],
        }
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_col{j}.json")
        with open(path, "w") as f:
            json.dump(out, f)
        print(name, j, e, out["iters_1e-8"], out["iters_1e-10"], round(out["seconds"]), flush=True)


if __name__ == "__main__":
    main()
