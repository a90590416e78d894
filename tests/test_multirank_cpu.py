"""The N > 1 path of bench.py on CPU: two gloo ranks, barrier, max over ranks.

Each rank runs its own replica (weak scaling); the job value uses the slowest rank's
time.  Runs as two spawned processes on 127.0.0.1 with the gloo backend.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.barrier(dist)
    ms = 10.0 * (rank + 1)                       # rank 1 is slower
    mx = bench.max_over_ranks(dist, ms, device="cpu")
    val = bench.job_value(100, world, mx)
    bench.barrier(dist)
    dist.destroy_process_group()
    q.put((rank, mx, val))


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert [r[1] for r in res] == [20.0, 20.0]          # both ranks see the max
    assert res[0][2] == pytest.approx(2 * 100 / 0.020)  # units of all ranks / slowest time


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.job_value(20, 1, 100.0) == pytest.approx(200.0)
