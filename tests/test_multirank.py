"""Multi-rank host logic of the benchmark on CPU (gloo, world sizes 2 and 8).

Columns are independent (Eq. TRACE-X-DECOMP of the paper), so ranks take
disjoint column batches and the only collectives are the max-over-ranks of
the step time and the sum of per-shift traces; all are checked here without
a GPU.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, n_chunks, n_batches, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_1609_08377_gb300 import sharding

    mine = sharding.stratified_batches(n_chunks, n_batches, rank, world, 0).tolist()
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    if rank == 0:
        out.put((gathered, t))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n_batches", [(2, 6), (8, 26)])
def test_ranks_disjoint_stratified_batches_and_max_time(world, n_batches):
    """The benchmark's batches: 16,384 columns in chunks of 32 (512 chunks);
    every rank gets n_batches distinct chunks spread over the whole
    longest-first order, no chunk twice across ranks; the job's step time is
    the slowest rank's."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n_chunks = 16384 // 32
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_chunks, n_batches, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, t = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t == 1.5 + (world - 1)
    seen = set()
    for mine in gathered:
        assert len(mine) == n_batches
        assert all(0 <= k < n_chunks for k in mine)
        # stratified: the rank's chunks span the order (first and last quarter both hit)
        assert min(mine) < n_chunks // 4 and max(mine) >= 3 * n_chunks // 4
        assert not (set(mine) & seen)
        seen |= set(mine)
    assert len(seen) == world * n_batches


def test_stratified_batches_refuse_reuse():
    from paper_1609_08377_gb300 import sharding

    with pytest.raises(ValueError):
        sharding.stratified_batches(100, 26, 0, 8)


# ---------------------------------------------------------------------------
# the one collective of the method: traces summed over ranks (Sec. III-C)
# ---------------------------------------------------------------------------

def _mu_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np

    from oracle import dense, density
    from paper_1609_08377_gb300 import sharding, synthetic as syn

    s = syn.make_system(64, 1.0, 0)
    eps = syn.energy_grid(32)
    w = syn.trapezoid_weights(eps)
    z = syn.shifts(eps, 0.2)
    cols_all = np.arange(s.M, dtype=np.int32)
    mine = sharding.shard_columns(cols_all, rank, world)
    G = dense.green_lu(s.A, s.B, z, mine)
    off = dense.pattern_offsets(s.A, mine)

    def trace_fn(cols):
        return density.shift_traces(G, s.B, cols, off)

    def mu_fn(sk, kT, n_elec, lo, hi):
        mu = density.find_mu(sk, eps, w, kT, n_elec, lo, hi)
        return mu, density.count_from_traces(sk, eps, w, mu, kT)

    n_full = density.count_from_traces(sharding.global_shift_traces(trace_fn, mine, dist), eps, w, 50.0, 0.2)
    mu, cnt = sharding.sharded_mu(trace_fn, mu_fn, mine, 0.2, 0.5 * n_full, -40.0, 40.0, dist)
    rho = density.density_from_green(G, eps, w, mu, 0.2)
    energy = sharding.sharded_trace(density.trace_with(rho, s.A, mine, off), dist)
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine.tolist(), mu, cnt, energy))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_chemical_potential_and_energy():
    """Columns split over 2 ranks; per-shift traces all-reduced: every rank
    gets the mu and energy of the single-process computation on all columns."""
    import numpy as np

    from oracle import dense, density
    from paper_1609_08377_gb300 import synthetic as syn

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_mu_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    # single process, all columns
    s = syn.make_system(64, 1.0, 0)
    eps = syn.energy_grid(32)
    w = syn.trapezoid_weights(eps)
    z = syn.shifts(eps, 0.2)
    cols = np.arange(s.M, dtype=np.int32)
    G = dense.green_lu(s.A, s.B, z, cols)
    off = dense.pattern_offsets(s.A, cols)
    sk = density.shift_traces(G, s.B, cols, off)
    n_full = density.count_from_traces(sk, eps, w, 50.0, 0.2)
    mu = density.find_mu(sk, eps, w, 0.2, 0.5 * n_full, -40.0, 40.0)
    energy = density.trace_with(density.density_from_green(G, eps, w, mu, 0.2), s.A, cols, off)
    seen = []
    for cols_r, mu_r, cnt_r, en_r in gathered:
        seen += cols_r
        assert abs(mu_r - mu) <= 1e-12 * max(1.0, abs(mu))
        assert abs(cnt_r - 0.5 * n_full) <= 1e-10 * n_full
        assert abs(en_r - energy) <= 1e-10 * abs(energy)
    assert sorted(seen) == list(range(s.M))
