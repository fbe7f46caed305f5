"""Bit-exactness at full size, on every workload, through the C ABI.

The serial oracle cannot mine the paper-scale (10^6 rows) or dense
(2*10^5 rows x 4,096 items) workloads in a test, so their results are pinned
by the negative-border certificate (tests/certificate.py): every single item
against np.bincount, every pair of frequent items (the whole pair border)
against direct pair counts, every larger itemset and every larger border
candidate against tid-list supports, downward closure -- which together hold
iff the result is exactly the set of frequent itemsets with their supports.
The first stops of the paper-scale loop are compared with the oracle's trace
row by row, and every autotuner configuration must give the same result.
"""
import numpy as np
import pytest

import oracle
import synth
from certificate import certify, item_counts, pair_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dic():
    import torch
    assert torch.cuda.is_available()
    import paper_1812_10959_gb300 as d
    return d


@pytest.fixture(scope="module")
def paper_scale():
    return synth.planted_paper_scale()


def test_paper_scale_certificate_every_configuration(dic, paper_scale):
    """The benchmark's workload (n=10^6, m=1,000, minsup 2,500, M=10^4): the
    library's rule and every configuration the autotuner may pick give the
    same itemsets and trace; the result passes the full certificate."""
    from paper_1812_10959_gb300 import autotune
    db = paper_scale
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    base = dic.mine(h, db.minsup, db.M)
    got = base.itemsets()
    for path, tw, form in autotune.CANDIDATES:
        r = dic.mine(h, db.minsup, db.M, path=path, tile_words=tw, count_form=form)
        assert r.itemsets() == got, (path, tw, form)
        assert r.trace.tolist() == base.trace.tolist(), (path, tw, form)
    h.free()
    info = certify(db.row_ptr, db.items, db.n, db.m, db.minsup, got)
    assert info["itemsets"] == 4091 and info["larger"] > 0 and info["pair_border"] > 400_000
    # the test count is m*n plus |DASHED| x block rows over the trace
    tr = base.trace.astype(np.int64)
    assert base.stats["tests"] == db.m * db.n + int((tr[:, 4] * (tr[:, 3] - tr[:, 2])).sum())


def test_paper_scale_first_stops_match_the_oracle_trace(dic, paper_scale):
    """Stops 1 and 2 of the paper-scale loop (498,501 pair circles counted
    over two blocks of 10^4 rows each) against the serial oracle."""
    db = paper_scale
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    res = dic.mine(h, db.minsup, db.M)
    h.free()
    ref = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M, max_stops=2,
                     superset_loop=False)
    assert len(ref.trace) == 2
    assert res.trace[:2].tolist() == ref.trace.tolist()


def test_dense_full_size_certificate(dic):
    """Dense workload at full size (2*10^5 rows, 4,096 items, minsup 20%,
    M=2*10^4): the TENSOR, BITSLICE, ROWS and automatic paths agree and the
    result passes the full certificate (all 150,000+ infrequent pairs of
    frequent items checked)."""
    db = synth.dense_zipf()
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    res = dic.mine(h, db.minsup, db.M)
    got = res.itemsets()
    for path in ("tensor", "bitslice", "rows"):
        r = dic.mine(h, db.minsup, db.M, path=path)
        assert r.itemsets() == got, path
        assert r.trace.tolist() == res.trace.tolist(), path
    h.free()
    info = certify(db.row_ptr, db.items, db.n, db.m, db.minsup, got)
    assert info["l1"] > 400 and info["pair_border"] > 100_000


def batched_sample():
    """Indices of the batched recipe's first 512 databases: the first six
    of every item count m, plus the largest database of every m (which
    includes the largest of all)."""
    by_m = {}
    for i in range(512):
        _, n, m, _, _, _ = synth.batched_params(i)
        by_m.setdefault(m, []).append((i, n))
    out = set()
    for m, v in by_m.items():
        out.update(i for i, _ in v[:6])
        out.add(max(v, key=lambda x: x[1])[0])
    return sorted(out)


def test_batched_sample_certificate(dic):
    """35 databases of the batched recipe (every m in {64,...,1024}, n up to
    ~2*10^5) mined together by dic_mine_batch: each result passes the full
    certificate; the small ones also match the oracle's trace."""
    idx = batched_sample()
    assert len(idx) >= 32
    dbs = [synth.batched_db(i) for i in idx]
    assert {d.m for d in dbs} == set(synth.BATCH_M_CHOICES)
    hs = [dic.load_db_csr(d.row_ptr, d.items, d.n, d.m) for d in dbs]
    res = dic.mine_batch(hs, [d.minsup for d in dbs], [d.M for d in dbs])
    for h in hs:
        h.free()
    traced = 0
    for d, r in zip(dbs, res):
        certify(d.row_ptr, d.items, d.n, d.m, d.minsup, r.itemsets())
        if d.n <= 20_000 and traced < 8:
            ref = oracle.dic(d.row_ptr, d.items, d.n, d.m, d.minsup, d.M, superset_loop=False)
            assert r.trace.tolist() == ref.trace.tolist()
            traced += 1
    assert traced >= 4


def test_served_paper_scale_databases_certificate(dic):
    """The two paper-scale databases of the served mix, queried through the
    request server (with small-database queries in the same mix) at
    thresholds and block sizes drawn from the served stream: every result
    passes the certificate and equals the query mined alone."""
    big = [synth.planted_paper_scale(seed=6000), synth.planted_paper_scale(seed=6001)]
    small = [synth.batched_db(i, base_seed=5000, n_hi=30_000) for i in range(6)]
    raw = small + big
    hs = [dic.load_db_csr(d.row_ptr, d.items, d.n, d.m) for d in raw]
    stream = synth.served_queries(4000, 66)
    qs, per_db = [], {64: 0, 65: 0}
    for q in stream:
        if q["db"] in per_db and per_db[q["db"]] < 3:
            per_db[q["db"]] += 1
            d = big[q["db"] - 64]
            qs.append((len(small) + q["db"] - 64, synth.minsup_count(d.n, q["frac"]),
                       max(1, d.n // q["mdiv"])))
        elif q["db"] < len(small) and len(qs) < 12:
            d = small[q["db"]]
            qs.append((q["db"], synth.minsup_count(d.n, q["frac"]), max(1, d.n // q["mdiv"])))
    assert sum(per_db.values()) == 6
    srv = dic.Server(max_slots=16)
    tickets = [srv.submit(hs[db], ms, M) for db, ms, M in qs]
    got = [srv.wait(t) for t in tickets]
    srv.close()
    pairs = {}
    for (db, ms, M), r in zip(qs, got):
        d = raw[db]
        if db >= len(small):
            if db not in pairs:
                lo = min(q[1] for q in qs if q[0] == db)
                cols = np.flatnonzero(item_counts(d.row_ptr, d.items, d.m) >= lo).tolist()
                pairs[db] = (cols, pair_matrix(d.row_ptr, d.items, d.n, d.m, cols))
            certify(d.row_ptr, d.items, d.n, d.m, ms, r.itemsets(), pairs=pairs[db])
        alone = dic.mine(hs[db], ms, M)
        assert r.itemsets() == alone.itemsets()
        assert r.trace.tolist() == alone.trace.tolist()
    for h in hs:
        h.free()
