"""Multi-process (replica) aggregation of the benchmark on CPU: two gloo ranks.

With N GPUs every rank mines its own copy of the database (the method has no
exchange step between independent mining jobs), so the whole-job figures are
the slowest rank's time and the sum of the ranks' tests. This checks that
reduction with world_size 2 over gloo, and that one process alone passes its
own figures through.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        # rank r: (r + 1) seconds and 1000 * (r + 1) tests
        t, n = bench.aggregate_replicas(float(rank + 1), 1000 * (rank + 1), "cpu")
        q.put((rank, t, n))
    finally:
        dist.destroy_process_group()


def test_single_process_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(2.5, 123, "cpu") == (2.5, 123.0)


def test_two_gloo_ranks_max_time_sum_tests():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n in got:
        assert t == 2.0          # the slowest rank's time
        assert n == 3000.0       # every rank's tests
