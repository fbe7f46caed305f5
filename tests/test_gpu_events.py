"""The event-driven stop loop against the per-stop loop and the oracle.

With every block staged and the pair cohort counted by the all-blocks GEMM,
each later cohort is counted over its whole pass when it is born; its
promotion and erase stops (Algorithm 4) are then known in advance and only
the stops that promote something run MAKECANDIDATES. The trace, the test
count and the result must be exactly those of Algorithm 2 run stop by stop.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dic():
    import torch
    assert torch.cuda.is_available()
    import paper_1812_10959_gb300 as d
    return d


def to_csr(rows):
    rp = np.zeros(len(rows) + 1, dtype=np.uint64)
    rp[1:] = np.cumsum([len(r) for r in rows])
    it = np.array([i for r in rows for i in r], dtype=np.uint32)
    return rp, it


def both_forms(dic, rp, it, n, m, minsup, M, **kw):
    db = dic.load_db_csr(rp, it, n, m)
    ev = dic.mine(db, minsup, M, path="tensor", stop_loop="events", **kw)
    ps = dic.mine(db, minsup, M, path="tensor", stop_loop="per-stop", **kw)
    db.free()
    assert ev.stats["event_loop"] == 1 and ps.stats["event_loop"] == 0
    assert ev.itemsets() == ps.itemsets()
    assert ev.trace.tolist() == ps.trace.tolist()
    assert ev.stats["tests"] == ps.stats["tests"]
    return ev, ps


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("M", [1, 3, 17, 100, 1000])
def test_random_databases_every_block_size(dic, seed, M):
    rp, it = synth.planted(seed=seed, n=600, m=40, n_patterns=25, pat_len_mean=4.0,
                           tx_len_mean=8.0)
    ev, _ = both_forms(dic, rp, it, 600, 40, 30, M)
    ref = oracle.dic(rp, it, 600, 40, 30, M, superset_loop=False)
    assert ev.itemsets() == ref.itemsets
    assert ev.trace.tolist() == ref.trace.tolist()
    assert ev.stats["tests"] == ref.tests
    # only stops with promotions cost an iteration
    assert 1 <= ev.stats["event_iters"] <= len(ref.trace) + 1


def test_planted_small_and_few_iterations(dic):
    db = synth.planted_small()
    ev, _ = both_forms(dic, db.row_ptr, db.items, db.n, db.m, db.minsup, db.M)
    ref = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M, superset_loop=False)
    assert ev.itemsets() == ref.itemsets
    assert ev.trace.tolist() == ref.trace.tolist()
    promoting = int((ref.trace[:, 5] > 0).sum())
    assert ev.stats["event_iters"] <= promoting + 1


def test_every_buffer_grows_inside_the_loop(dic):
    """minsup = n over rows sharing 15 items: the candidate store, the box set
    and the trace (about 15 full passes of 6 blocks) all outgrow their first
    sizes while the loop runs; every subset of the shared items has support n."""
    core = list(range(3, 18))
    rng = np.random.default_rng(9)
    rows = [core + rng.integers(20, 60, 3).tolist() for _ in range(40)]
    rp, it = to_csr(rows)
    ev, _ = both_forms(dic, rp, it, 40, 60, 40, 7)
    got = ev.itemsets()
    assert len(got) == 2 ** 15 - 1
    assert all(s == 40 and set(x) <= set(core) for x, s in got)
    assert len(ev.trace) > 64  # beyond the first trace capacity


def test_itemsets_longer_than_the_stored_ranks(dic):
    """Itemsets of up to 17 items (a record stores 16 ranks): the cohort pass
    reads them from the record's mask. Closed form: minsup = n over rows that
    share 17 items gives every non-empty subset of them, support n."""
    core = list(range(17))
    rows = [core + [17 + (t % 5)] for t in range(30)]
    rp, it = to_csr(rows)
    db = dic.load_db_csr(rp, it, 30, 24)
    ev = dic.mine(db, 30, 10, path="tensor", stop_loop="events")
    db.free()
    assert ev.stats["event_loop"] == 1
    got = ev.itemsets()
    assert len(got) == 2 ** 17 - 1
    assert max(len(x) for x, _ in got) == 17
    assert all(s == 30 for _, s in got)


def test_profiled_segments_equal_one_graph(dic):
    """Timing the cohort pass on one iteration in three (graph segments with
    direct launches between them) changes nothing in the result or trace."""
    db = synth.planted_small()
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    kw = dict(path="tensor", stop_loop="events")
    a = dic.mine(h, db.minsup, db.M, **kw)
    b = dic.mine(h, db.minsup, db.M, profile=["count", "gen"], profile_every=3, **kw)
    c = dic.mine(h, db.minsup, db.M, use_graph=False, **kw)
    assert a.stats["event_loop"] == b.stats["event_loop"] == c.stats["event_loop"] == 1
    h.free()
    assert a.itemsets() == b.itemsets() == c.itemsets()
    assert a.trace.tolist() == b.trace.tolist() == c.trace.tolist()
    assert b.stats["count_launches"] >= 1 and b.stats["count_ops_timed"] > 0


def test_dense_reduced_rows(dic):
    db = synth.dense_zipf(n=2000)
    ev, _ = both_forms(dic, db.row_ptr, db.items, db.n, db.m, db.minsup, 400)
    ref = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, 400, superset_loop=False)
    assert ev.itemsets() == ref.itemsets
    assert ev.trace.tolist() == ref.trace.tolist()


@pytest.mark.parametrize("seed", [0, 1])
def test_hand_over_from_the_per_stop_loop(dic, seed):
    """stop_loop "auto": the per-stop loop hands the rest of the loop to the
    event-driven form once the pair cohort has passed and promotions have
    stopped; the live records are counted over the blocks left of their
    passes from their counts so far. Result, trace and test count equal the
    per-stop loop's and the oracle's."""
    rp, it = synth.planted(seed=seed, n=4000, m=60, n_patterns=40, pat_len_mean=4.0,
                           tx_len_mean=9.0)
    n, m, minsup, M = 4000, 60, 60, 40   # 100 blocks
    db = dic.load_db_csr(rp, it, n, m)
    au = dic.mine(db, minsup, M, path="tensor")
    ps = dic.mine(db, minsup, M, path="tensor", stop_loop="per-stop")
    # profiling times the per-stop stops only and changes nothing
    pr = dic.mine(db, minsup, M, path="tensor", profile=["count", "gen"], profile_every=3)
    db.free()
    assert pr.stats["event_loop"] == 2
    assert pr.itemsets() == au.itemsets() and pr.trace.tolist() == au.trace.tolist()
    assert pr.stats["count_launches"] >= 1 and pr.stats["count_ops_timed"] > 0
    ref = oracle.dic(rp, it, n, m, minsup, M, superset_loop=False)
    assert au.stats["event_loop"] == 2 and ps.stats["event_loop"] == 0
    assert au.itemsets() == ps.itemsets() == ref.itemsets
    assert au.trace.tolist() == ps.trace.tolist() == ref.trace.tolist()
    assert au.stats["tests"] == ps.stats["tests"] == ref.tests
