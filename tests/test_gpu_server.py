"""The request server (dic_server_*): queries that arrive while others run
are admitted as slots and memory free up and advance together; each result
must be exactly the one the query gets alone (and the oracle's, for the
small databases)."""
import threading

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dic():
    import paper_1812_10959_gb300 as d
    return d


@pytest.fixture(scope="module")
def dbs(dic):
    raw = [synth.batched_db(i, base_seed=5000, n_hi=30_000) for i in range(10)]
    raw.append(synth.planted_small())
    hs = [dic.load_db_csr(d.row_ptr, d.items, d.n, d.m) for d in raw]
    yield raw, hs
    for h in hs:
        h.free()


def queries(raw, count, seed=11):
    out = []
    for i, q in enumerate(synth.served_queries(count, len(raw), seed=seed)):
        d = raw[q["db"]]
        out.append((q["db"], synth.minsup_count(d.n, max(q["frac"], 0.01)), max(1, d.n // q["mdiv"])))
    return out


def test_results_same_alone_and_in_the_mix(dic, dbs):
    raw, hs = dbs
    qs = queries(raw, 60)
    srv = dic.Server(max_slots=16)
    tickets = []
    lock = threading.Lock()

    def submitter(part):
        for i in part:
            t = srv.submit(hs[qs[i][0]], qs[i][1], qs[i][2])
            with lock:
                tickets.append((i, t))

    threads = [threading.Thread(target=submitter, args=(range(k, len(qs), 3),)) for k in range(3)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    got = {i: srv.wait(t) for i, t in tickets}
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(qs)
    assert st["peak_slots"] > 1          # their work overlapped on the device
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for i, (db, minsup, M) in enumerate(qs):
        alone = dic.mine(hs[db], minsup, M)
        assert got[i].itemsets() == alone.itemsets()
        assert got[i].trace.tolist() == alone.trace.tolist()
    checked = 0
    for i, (db, minsup, M) in enumerate(qs):
        d = raw[db]
        if d.n <= 8000 and d.m <= 128 and checked < 4:
            ref = oracle.dic(d.row_ptr, d.items, d.n, d.m, minsup, M)
            assert got[i].itemsets() == ref.itemsets
            checked += 1


def test_tight_budget_admits_one_query_at_a_time(dic, dbs):
    raw, hs = dbs
    qs = queries(raw, 8, seed=3)
    srv = dic.Server(hbm_budget_bytes=1, max_slots=8)
    ts = [srv.submit(hs[db], ms, M) for db, ms, M in qs]
    res = [srv.wait(t) for t in ts]
    st = srv.stats()
    srv.close()
    assert st["peak_slots"] <= 1
    for (db, ms, M), r in zip(qs, res):
        assert r.itemsets() == dic.mine(hs[db], ms, M).itemsets()


def test_server_errors(dic, dbs):
    raw, hs = dbs
    srv = dic.Server(max_slots=2)
    with pytest.raises(dic.DicError):
        srv.wait(12345)
    with pytest.raises(dic.DicError):
        srv.submit(hs[0], 0, 10)
    t = srv.submit(hs[0], raw[0].minsup, raw[0].M)
    assert srv.wait(t).itemsets() == dic.mine(hs[0], raw[0].minsup, raw[0].M).itemsets()
    with pytest.raises(dic.DicError):
        srv.wait(t)                      # a ticket is waited once
    srv.close()


def test_large_databases_are_mined_alone_beside_the_rounds(dic, dbs):
    """With solo_rows below some databases' size, their queries take no slot:
    each is mined alone by the single-query path beside the batched rounds.
    Every result still equals the query mined alone."""
    raw, hs = dbs
    qs = queries(raw, 40, seed=21)
    srv = dic.Server(max_slots=8, solo_rows=8000)
    ts = [srv.submit(hs[db], ms, M) for db, ms, M in qs]
    got = [srv.wait(t) for t in ts]
    st = srv.stats()
    srv.close()
    big = sum(1 for db, _, _ in qs if raw[db].n >= 8000)
    assert 0 < big < len(qs)
    assert st["solo"] == big and st["completed"] == len(qs)
    for (db, ms, M), r in zip(qs, got):
        alone = dic.mine(hs[db], ms, M)
        assert r.itemsets() == alone.itemsets()
        assert r.trace.tolist() == alone.trace.tolist()
