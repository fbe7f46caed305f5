"""Association rules on the GPU (dic_rules_from_itemsets) against the
oracle's rules, on mined itemsets and on hand-built inputs; error cases."""
import numpy as np
import pytest

import oracle
import synth
from golden_io import to_csr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dic():
    import torch
    assert torch.cuda.is_available()
    import paper_1812_10959_gb300 as d
    return d


@pytest.mark.parametrize("seed", range(4))
def test_rules_random_small(dic, seed):
    rng = np.random.default_rng(7100 + seed)
    m = int(rng.integers(2, 130))
    n = int(rng.integers(1, 300))
    p = 0.4 if m < 20 else 0.08
    rows = [np.flatnonzero(rng.random(m) < p).tolist() for _ in range(n)]
    rp, it = to_csr(rows)
    minsup = max(1, n // 10)
    db = dic.load_db_csr(rp, it, n, m)
    res = dic.mine(db, minsup, max(1, n // 3))
    ref_L = oracle.dic(rp, it, n, m, minsup, max(1, n // 3)).itemsets
    for num, den in ((0, 1), (1, 2), (3, 4), (1, 1)):
        assert dic.rules(res, num, den, m=m) == oracle.rules(ref_L, num, den)
    db.free()


def test_rules_planted_small(dic):
    db = synth.planted_small(1)
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    res = dic.mine(h, db.minsup, db.M)
    ref_L = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M).itemsets
    for num, den in ((1, 5), (1, 3), (1, 2)):  # 630, 156 and 15 rules
        got = dic.rules(res, num, den, m=db.m)
        assert got == oracle.rules(ref_L, num, den)
        assert len(got) > 10
    h.free()


def test_rules_word_boundaries(dic):
    # items 63, 64, 127, 128 in one itemset family across words
    rows = [[0, 63, 64, 127, 128], [63, 64, 128], [0, 63, 64, 127, 128], [63, 127]] * 5
    rp, it = to_csr(rows)
    n, m = len(rows), 130
    db = dic.load_db_csr(rp, it, n, m)
    res = dic.mine(db, 5, 7)
    ref_L = oracle.dic(rp, it, n, m, 5, 7).itemsets
    assert dic.rules(res, 1, 2, m=m) == oracle.rules(ref_L, 1, 2)
    db.free()


def test_rules_errors(dic):
    from paper_1812_10959_gb300.dic import Result
    W = 1
    masks = np.array([[0b11]], dtype=np.uint64)  # {0, 1} without its subsets
    res = Result(W, masks, np.array([2], dtype=np.uint32), np.array([5], dtype=np.uint32),
                 np.zeros((0, 9), dtype=np.uint64), {})
    with pytest.raises(dic.DicError):
        dic.rules(res, 1, 2, m=2)   # not downward closed
    with pytest.raises(dic.DicError):
        dic.rules(res, 1, 0, m=2)   # conf_den = 0
    bad = Result(W, masks, np.array([3], dtype=np.uint32), np.array([5], dtype=np.uint32),
                 np.zeros((0, 9), dtype=np.uint64), {})
    with pytest.raises(dic.DicError):
        dic.rules(bad, 1, 2, m=2)   # size is not the popcount
    empty = Result(W, np.zeros((0, 1), dtype=np.uint64), np.zeros(0, dtype=np.uint32),
                   np.zeros(0, dtype=np.uint32), np.zeros((0, 9), dtype=np.uint64), {})
    assert dic.rules(empty, 1, 2, m=2) == []
