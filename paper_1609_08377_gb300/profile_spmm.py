"""Small, fixed workloads for profiling the solver's kernels.

    python -m paper_1609_08377_gb300.profile_spmm spmm  --atoms 100000 --w 64 --reps 3
    python -m paper_1609_08377_gb300.profile_spmm solve --atoms 20000 --w 64 --steps 6

`spmm` runs `reps` applications of the inner-CG product Y = B X (FP32, the
fused CG form) on the seeded C/H pencil; with --time it also prints the mean
duration per launch from CUDA events over 20 more launches and the
algorithmic bytes per launch. `solve` runs a short host-driven solve (no
CUDA graph, so a profiler sees every kernel) of 64 seeded columns with 128
shifts in the double-float mixed mode, truncated at `steps` Lanczos steps.
Both print "ok" on success.
"""

from __future__ import annotations

import argparse

import numpy as np

from . import synthetic as syn


def spmm_alg_bytes(s, n_blocks: int, W: int, bv: int = 4) -> int:
    """Algorithmic bytes of one fused CG product on W lanes of bv-byte values:
    the stored values once, one neighbour index per atom block, the atom
    pointers, X read once, and the direction P and the product Y each read
    and written once."""
    return s.nnz * bv + n_blocks * 4 + (s.n_atoms + 1) * 4 + 5 * s.M * W * bv


def atom_blocks(s) -> int:
    """Atom blocks of A: the number of (atom, neighbour atom) pairs, the
    neighbour index entries of the block layout before padding."""
    atom = s.atom_of_row()
    A = s.A
    cnt = 0
    for I in range(s.n_atoms):
        row = int(s.orb_offset[I])
        cnt += np.unique(atom[A.indices[A.indptr[row]:A.indptr[row + 1]]]).size
    return cnt


def main(argv=None) -> None:
    import torch

    from . import gsk

    ap = argparse.ArgumentParser()
    ap.add_argument("mode", choices=["spmm", "solve"])
    ap.add_argument("--atoms", type=int, default=20000)
    ap.add_argument("--w", type=int, default=64)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--time", action="store_true")
    a = ap.parse_args(argv)
    s = syn.make_system(a.atoms, 1.0 / 3.0, 0)
    solver = gsk.from_system(s)
    if a.mode == "spmm":
        X = torch.randn(s.M * a.w, device="cuda")
        Y = torch.empty_like(X)
        solver.spmm(1, gsk.GSK_MIXED, a.w, X, Y, n_rep=a.reps)
        torch.cuda.synchronize()
        if a.time:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            solver.spmm(1, gsk.GSK_MIXED, a.w, X, Y, n_rep=20)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 20
            alg = spmm_alg_bytes(s, atom_blocks(s), a.w)
            print(f"atoms={a.atoms} M={s.M} W={a.w}: {ms * 1e3:.1f} us per launch, "
                  f"{alg / 1e6:.1f} MB algorithmic, {alg / ms / 1e6:.0f} GB/s")
    else:
        z = syn.shifts(syn.energy_grid(128), 0.1)
        cols = syn.column_subset(s.M, 64, 0)
        off = solver.pattern_offsets(cols)
        G = torch.zeros(int(off[-1]) * z.size, dtype=torch.complex128, device="cuda")
        solver.solve(z, cols, G, precision="mixed_df", batch_w=a.w, tol=1e-8, max_iter=a.steps, use_graph=0)
        torch.cuda.synchronize()
    solver.close()
    print("ok")


if __name__ == "__main__":
    main()
