"""Transaction-sharded counting with one sum of the counters per stop (the
data-distributed scheme of the paper's related work), on CPU ranks: two gloo
ranks each count their half of every block with the multi-core CPU program
(oracle/paralleldic_omp.cpp), sum the first-pass and per-stop counters with
torch.distributed.all_reduce, run the lattice steps on the totals, and must
each return exactly the single-rank oracle's itemsets, supports, per-stop
trace and test count. This is the seam a multi-GPU form would use (one
all-reduce of the dashed itemsets' counters per stop); it is not measured on
GPUs here."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _cases():
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import numpy as np
    import synth
    from golden_io import to_csr
    db = synth.planted_small()
    out = [(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M),
           (db.row_ptr, db.items, db.n, db.m, db.minsup, 777)]
    rng = np.random.default_rng(4)
    rows = [np.flatnonzero(rng.random(20) < 0.3).tolist() for _ in range(97)]
    rp, it = to_csr(rows)
    out.append((rp, it, 97, 20, 9, 13))       # blocks split unevenly; a ragged tail
    out.append((rp, it, 97, 20, 9, 1))        # one-row blocks: one rank counts nothing
    return out


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    calls = [0]

    def reduce(counts):
        t = torch.from_numpy(counts.view("int64"))
        dist.all_reduce(t)
        calls[0] += 1

    try:
        out = []
        for rp, it, n, m, minsup, M in _cases():
            r, _ = oracle.paralleldic_sharded(rp, it, n, m, minsup, M, rank, world, reduce,
                                              threads=2)
            out.append((r.itemsets, r.trace.tolist(), r.tests))
        q.put((rank, out, calls[0]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_oracle():
    mp = pytest.importorskip("torch.multiprocessing")
    sys.path.insert(0, ROOT)
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    refs = [oracle.dic(rp, it, n, m, minsup, M) for rp, it, n, m, minsup, M in _cases()]
    for rank, out, calls in got:
        # one reduce for the first pass and one per stop of every case
        assert calls == sum(1 + len(ref.trace) for ref in refs)
        for (items, trace, tests), ref in zip(out, refs):
            assert items == ref.itemsets
            assert trace == ref.trace.tolist()
            assert tests == ref.tests


def test_one_rank_is_the_unsharded_program():
    sys.path.insert(0, ROOT)
    import oracle
    for rp, it, n, m, minsup, M in _cases():
        a, _ = oracle.paralleldic_sharded(rp, it, n, m, minsup, M, 0, 1, None, threads=2)
        b, _ = oracle.paralleldic(rp, it, n, m, minsup, M, threads=2)
        assert a.itemsets == b.itemsets and a.trace.tolist() == b.trace.tolist()
