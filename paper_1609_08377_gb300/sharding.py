"""Column sharding over ranks and the one collective of the method.

Columns are independent (Eq. TRACE-X-DECOMP): each rank solves its own
columns and keeps its G and rho. The only exchange is the sum of trace
quantities over all columns (the paper's MPI_Allreduce of Sec. III-C): the
electron count that fixes the chemical potential, the energy, and other
Tr(rho X). Summing the S per-shift traces s_k instead of a scalar lets every
rank search mu on the global count with one all-reduce of S numbers:

    N(mu) = -(1/pi) sum_k w_k f_mu(e_k) sum_ranks s_k(rank)

The functions take the per-rank trace and search steps as callables, so the
same code runs with the library's kernels (Solver.shift_trace,
Solver.mu_from_traces) on GPUs under NCCL, or with any other implementation
of those two steps on CPU ranks under gloo.
"""

from __future__ import annotations

import numpy as np


def shard_columns(cols, rank: int, world: int) -> np.ndarray:
    """Columns of this rank: every world-th column starting at rank, so a
    column order that is longest-first (the learned scheduler's) stays
    balanced across ranks."""
    cols = np.asarray(cols, dtype=np.int32)
    return np.ascontiguousarray(cols[rank::world])


def stratified_batches(n_chunks: int, n_take: int, rank: int, world: int, seed: int = 0) -> np.ndarray:
    """Batch (chunk) indices of this rank for a benchmark over a column set
    cut into n_chunks chunks of consecutive columns (in the learned scheduler's
    longest-first order): n_take * world indices evenly spaced over
    [0, n_chunks), dealt to the ranks round-robin, so every rank gets a
    stratified sample of the set and no chunk is used twice as long as
    n_take * world <= n_chunks; then shuffled (seeded) within the rank, so the
    first (warm-up) batches are not all of one kind."""
    total = n_take * world
    if total > n_chunks:
        raise ValueError(f"{n_take} batches on {world} ranks need {total} chunks; the set has {n_chunks}")
    idx = np.floor((np.arange(total) + 0.5) * n_chunks / total).astype(np.int64)
    mine = idx[rank::world]
    rng = np.random.default_rng(seed + 1000 + rank)
    return mine[rng.permutation(mine.size)]


def allreduce_sum(x, dist=None, device="cpu") -> np.ndarray:
    """Sum of a host vector over all ranks (identity without a process group).
    The sum runs in FP64 on `device` (a CUDA device under NCCL)."""
    x = np.asarray(x, dtype=np.float64)
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x.copy()
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x)).to(device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.cpu().numpy()


def global_shift_traces(trace_fn, cols_local, dist=None, device="cpu") -> np.ndarray:
    """s_k summed over every rank's columns; trace_fn(cols) returns the S
    per-shift traces of the given local columns (host array)."""
    return allreduce_sum(trace_fn(cols_local), dist, device)


def sharded_mu(trace_fn, mu_fn, cols_local, kT: float, n_elec: float, mu_lo: float, mu_hi: float, dist=None,
               device="cpu"):
    """Chemical potential for n_elec electrons over the whole column set.
    mu_fn(s, kT, n_elec, lo, hi) -> (mu, N(mu)) searches on global traces; every
    rank gets the same mu."""
    s = global_shift_traces(trace_fn, cols_local, dist, device)
    return mu_fn(s, kT, n_elec, mu_lo, mu_hi)


def sharded_trace(local_value: float, dist=None, device="cpu") -> float:
    """A scalar trace (Tr rho X over the local columns) summed over all ranks."""
    return float(allreduce_sum(np.array([local_value]), dist, device)[0])
