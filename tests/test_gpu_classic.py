"""Classic DIC (Algorithm 1: no first pass, every 1-itemset starts as a dashed
circle) on the GPU against the oracle's classic DIC: itemsets, supports, the
per-stop trace and the test count; and the same itemsets as ParallelDIC."""
import math

import numpy as np
import pytest

import oracle
import synth
from golden_io import hand_examples, to_csr

pytestmark = pytest.mark.gpu
PATHS = ["rows", "bitslice", "auto"]


@pytest.fixture(scope="module")
def dic():
    import torch
    assert torch.cuda.is_available()
    import paper_1812_10959_gb300 as d
    return d


def check(dic, rp, it, n, m, minsup, M, path):
    db = dic.load_db_csr(rp, it, n, m)
    res = dic.mine(db, minsup, M, path=path, algorithm="classic")
    ref = oracle.dic_classic(rp, it, n, m, minsup, M)
    assert res.itemsets() == ref.itemsets
    assert res.trace.tolist() == ref.trace.tolist()
    assert res.stats["tests"] == ref.tests
    db.free()
    return res, ref


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("ex", hand_examples(), ids=lambda e: e["name"])
def test_hand_examples_classic(dic, ex, path):
    rp, it = to_csr(ex["rows"])
    res, _ = check(dic, rp, it, ex["n"], ex["m"], ex["minsup"], ex["M"], path)
    assert res.itemsets() == ex["L"]  # the same L as ParallelDIC


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("seed", range(4))
def test_random_small_classic(dic, seed, path):
    rng = np.random.default_rng(900 + seed)
    m = int(rng.integers(1, 100))
    n = int(rng.integers(1, 300))
    p = float(rng.uniform(0.05, 0.4)) if m < 40 else float(rng.uniform(0.02, 0.1))
    rows = [np.flatnonzero(rng.random(m) < p).tolist() for _ in range(n)]
    rp, it = to_csr(rows)
    for minsup in sorted({max(2, n // 20), max(1, n // 8), n}):
        for M in sorted({1, 3, math.ceil(n / 3), n}):
            res, _ = check(dic, rp, it, n, m, minsup, M, path)
            assert res.itemsets() == oracle.dic(rp, it, n, m, minsup, M).itemsets


def test_planted_small_classic(dic):
    db = synth.planted_small(2)
    res, ref = check(dic, db.row_ptr, db.items, db.n, db.m, db.minsup, db.M, "auto")
    assert len(ref.itemsets) > 100
    par = dic.mine(dic.load_db_csr(db.row_ptr, db.items, db.n, db.m), db.minsup, db.M)
    assert par.itemsets() == res.itemsets()


def test_classic_rejected_in_batches(dic):
    db = synth.planted_small(0)
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    with pytest.raises(dic.DicError):
        dic.mine_batch([h], [db.minsup], [db.M], algorithm="classic")
    h.free()
