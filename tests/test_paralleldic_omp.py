"""The multi-core CPU baseline (oracle/paralleldic_omp.cpp: ParallelDIC with
OpenMP, the paper's own parallel design) returns exactly the oracle's
itemsets, supports, per-stop trace and test count, at every thread count,
including the nested balancing of Figure 3 (fewer dashed itemsets than
threads)."""
import math

import numpy as np
import pytest

import oracle
import synth
from golden_io import hand_examples, to_csr


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_equals_the_oracle_on_the_planted_small_workload(threads):
    db = synth.planted_small()
    ref = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M)
    got, used = oracle.paralleldic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M,
                                   threads=threads)
    assert used == threads
    assert got.itemsets == ref.itemsets
    assert got.trace.tolist() == ref.trace.tolist()
    assert got.tests == ref.tests


@pytest.mark.parametrize("seed", range(6))
def test_equals_the_oracle_on_random_databases_every_M(seed):
    rng = np.random.default_rng(900 + seed)
    m = int(rng.integers(2, 90))
    n = int(rng.integers(1, 300))
    p = float(rng.uniform(0.05, 0.4)) if m < 30 else float(rng.uniform(0.03, 0.12))
    rows = [np.flatnonzero(rng.random(m) < p).tolist() for _ in range(n)]
    rp, it = to_csr(rows)
    for minsup in sorted({max(1, n // 10), max(1, n // 4), n}):
        for M in sorted({1, 7, math.ceil(n / 3), n, n + 3}):
            ref = oracle.dic(rp, it, n, m, minsup, M)
            got, _ = oracle.paralleldic(rp, it, n, m, minsup, M, threads=8)
            assert got.itemsets == ref.itemsets
            assert got.trace.tolist() == ref.trace.tolist()


def test_hand_worked_examples():
    for ex in hand_examples():
        rp, it = to_csr(ex["rows"])
        got, _ = oracle.paralleldic(rp, it, ex["n"], ex["m"], ex["minsup"], ex["M"], threads=4)
        assert got.itemsets == ex["L"]
        assert got.trace.tolist() == ex["trace"]
        assert got.tests == ex["tests"]


def test_bounded_sample_stops_after_max_stops():
    db = synth.planted_small()
    got, _ = oracle.paralleldic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M, max_stops=2)
    ref = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M, max_stops=2)
    assert got.trace.tolist() == ref.trace.tolist()
    assert got.tests == ref.tests
