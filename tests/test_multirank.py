"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

Columns are independent (Eq. TRACE-X-DECOMP of the paper), so ranks take
disjoint column batches and the only collective is the max-over-ranks of the
step time; both are checked here without a GPU.
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


def _worker(rank, world, port, n_cols, C, n_batches, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ranges = bench.rank_batches(n_cols, C, n_batches, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, ranges)
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    if rank == 0:
        out.put((gathered, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_batches_and_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    n_cols, C, n_batches = 8192, 128, 6
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_cols, C, n_batches, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, t = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t == 2.5
    seen = set()
    for ranges in gathered:
        assert len(ranges) == n_batches
        for a, b in ranges:
            assert b - a == C
            cols = set(range(a, b))
            assert not (cols & seen)
            seen |= cols
    assert len(seen) == 2 * n_batches * C
