"""Batched mining (dic_mine_batch): many independent databases advance one
stop per round with one launch per phase for all of them. Every query's
result must be exactly what the oracle (small databases) and the single-query
path give, whatever else is in the batch."""
import numpy as np
import pytest

import oracle
import synth
from golden_io import to_csr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dic():
    import paper_1812_10959_gb300 as d
    return d


def mixed_queries():
    """Small and uneven databases, including degenerate ones."""
    qs = []
    rng = np.random.default_rng(42)
    for i in range(14):
        m = int(rng.choice([20, 64, 100, 130, 300]))
        n = int(rng.integers(300, 2500))
        rp, it = synth.planted(100 + i, n, m, 2 * m, float(rng.uniform(2, 6)),
                               min(float(rng.uniform(4, 14)), m / 6))
        minsup = max(6, int(n * rng.uniform(0.02, 0.05)))
        M = int(rng.integers(1, n + 10))
        qs.append((rp, it, n, m, minsup, M))
    qs.append(to_csr([]) + (0, 8, 1, 3))                 # empty database
    qs.append(to_csr([[1], [2], [1]]) + (3, 8, 2, 2))    # one frequent item, no pairs
    qs.append(to_csr([list(range(12))] * 6) + (6, 16, 6, 4))   # deep lattice, growth
    return qs


def test_batch_equals_oracle_and_single(dic):
    qs = mixed_queries()
    dbs = [dic.load_db_csr(rp, it, n, m) for rp, it, n, m, _, _ in qs]
    res = dic.mine_batch(dbs, [q[4] for q in qs], [q[5] for q in qs])
    for (rp, it, n, m, minsup, M), db, r in zip(qs, dbs, res):
        ref = oracle.dic(rp, it, n, m, minsup, M)
        assert r.itemsets() == ref.itemsets
        assert r.trace.tolist() == ref.trace.tolist()
        assert r.stats["tests"] == ref.tests
        single = dic.mine(db, minsup, M)
        assert single.itemsets() == r.itemsets()
    for db in dbs:
        db.free()


def test_batch_same_db_several_queries(dic):
    """One database shared by queries with different minsup and M."""
    db0 = synth.planted_small()
    h = dic.load_db_csr(db0.row_ptr, db0.items, db0.n, db0.m)
    params = [(200, 1000), (150, 777), (300, 10_000), (120, 333), (200, 1)]
    res = dic.mine_batch([h] * len(params), [p[0] for p in params], [p[1] for p in params])
    for (minsup, M), r in zip(params, res):
        ref = oracle.dic(db0.row_ptr, db0.items, db0.n, db0.m, minsup, M)
        assert r.itemsets() == ref.itemsets
        assert r.trace.tolist() == ref.trace.tolist()
    h.free()


def test_batched_recipe_subset(dic):
    """Databases of the batched recipe (uneven n and m): batch == single."""
    dbs = [synth.batched_db(i, n_hi=20_000) for i in range(24)]
    hs = [dic.load_db_csr(d.row_ptr, d.items, d.n, d.m) for d in dbs]
    res = dic.mine_batch(hs, [d.minsup for d in dbs], [d.M for d in dbs])
    for d, h, r in zip(dbs, hs, res):
        s = dic.mine(h, d.minsup, d.M)
        assert s.itemsets() == r.itemsets()
        assert s.trace.tolist() == r.trace.tolist()
    small = [i for i, d in enumerate(dbs) if d.n <= 8000 and d.m <= 128][:4]
    for i in small:
        d = dbs[i]
        ref = oracle.dic(d.row_ptr, d.items, d.n, d.m, d.minsup, d.M)
        assert res[i].itemsets() == ref.itemsets
    for h in hs:
        h.free()


def test_plain_per_query_path_equals_batch(dic):
    qs = mixed_queries()[:6]
    dbs = [dic.load_db_csr(rp, it, n, m) for rp, it, n, m, _, _ in qs]
    a = dic.mine_batch(dbs, [q[4] for q in qs], [q[5] for q in qs])
    b = dic.mine_batch(dbs, [q[4] for q in qs], [q[5] for q in qs], path="rows")
    assert [r.itemsets() for r in a] == [r.itemsets() for r in b]
    for db in dbs:
        db.free()
