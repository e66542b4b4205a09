"""A fixed multiple Arnoldi workload for profiling (64 seeded columns of the
seeded C/H pencil, nu = 30, rho only):

    python -m paper_1609_08377_gb300.profile_ma --atoms 20000

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
    ap.add_argument("--cols", type=int, default=64)
    ap.add_argument("--nu", type=int, default=30)
    a = ap.parse_args(argv)
    s = syn.make_system(a.atoms, 1.0 / 3.0, 0)
    solver = gsk.from_system(s)
    cols = syn.column_subset(s.M, a.cols, 0)
    off = solver.pattern_offsets(cols)
    rho = torch.zeros(int(off[-1]), dtype=torch.float64, device="cuda")
    solver.marnoldi(cols, a.nu, -10.0, 0.1, rho)
    torch.cuda.synchronize()
    solver.close()
    print("ok")


if __name__ == "__main__":
    main()
