"""The N>1 path of bench.py on the CPU: two ranks over gloo (127.0.0.1).

Independent problems shard with no data-path collective; the only
collectives are the barrier around the timed region and the max over ranks
of the timed duration.  This checks that host logic with world_size 2.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    w, r, local = bench.dist_init()
    v = bench.max_over_ranks(1.5 * (r + 1), w)
    bench.barrier(w)
    q.put((r, w, local, v))
    dist.destroy_process_group()


def test_max_over_ranks_and_barrier_with_two_gloo_ranks():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert results == [(0, 2, 0, 3.0), (1, 2, 1, 3.0)]


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(2.5, 1) == 2.5
    bench.barrier(1)
