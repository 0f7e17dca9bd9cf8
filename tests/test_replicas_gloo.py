"""Multi-process path of bench.py (independent replicas, one per GPU) on CPU:
two gloo ranks reduce their timings and work the way the benchmark does
(slowest rank's time, summed work)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = 100.0 + 50.0 * rank
        solve_ms = 80.0 + 10.0 * rank
        work = 1e9 * (rank + 1)
        q.put((rank, bench.reduce_over_ranks(dist, step_ms, solve_ms, work, "cpu")))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (150.0, 90.0, 3e9)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, 1.0, 2.0, 3.0, "cpu") == (1.0, 2.0, 3.0)
