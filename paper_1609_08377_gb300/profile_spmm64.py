"""The FP64 block SpMM on 64 lanes (the multiple Arnoldi path's A-product),
for profiling:

    python -m paper_1609_08377_gb300.profile_spmm64 --atoms 20000 --reps 3

Prints "ok" on success.
"""

from __future__ import annotations

import argparse


def main(argv=None) -> None:
    import torch

    from . import gsk
    from . import synthetic as syn

    ap = argparse.ArgumentParser()
    ap.add_argument("--atoms", type=int, default=20000)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    s = syn.make_system(a.atoms, 1.0 / 3.0, 0)
    solver = gsk.from_system(s)
    X = torch.randn(s.M * 64, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    solver.spmm(0, gsk.GSK_FP64, 64, X, Y, n_rep=a.reps)
    torch.cuda.synchronize()
    solver.close()
    print("ok")


if __name__ == "__main__":
    main()
