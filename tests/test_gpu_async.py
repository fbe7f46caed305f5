"""dic_mine_async / dic_mine_wait through the C ABI: two mines started on
two streams overlap and each returns the oracle's itemsets, supports and
trace; a wait with a short limit on a running mine times out and the job
can still be waited afterwards."""
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dic():
    import paper_1812_10959_gb300 as d
    return d


def test_two_mines_on_two_streams_match_the_oracle(dic):
    import torch
    a = synth.planted_small()
    rp, it = synth.planted(seed=5, n=3000, m=70, n_patterns=60, pat_len_mean=4.0,
                           tx_len_mean=9.0)
    b = synth.Database("b", 3000, 70, rp, it, 60, 700)
    ha = dic.load_db_csr(a.row_ptr, a.items, a.n, a.m)
    hb = dic.load_db_csr(b.row_ptr, b.items, b.n, b.m)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    jobs = [dic.mine_async(ha, a.minsup, a.M, stream=s1),
            dic.mine_async(hb, b.minsup, b.M, stream=s2),
            dic.mine_async(ha, a.minsup, 333, stream=s2, path="rows")]
    res = [j.wait() for j in jobs]
    for (d, M), r in zip(((a, a.M), (b, b.M), (a, 333)), res):
        ref = oracle.dic(d.row_ptr, d.items, d.n, d.m, d.minsup, M)
        assert r.itemsets() == ref.itemsets
        assert r.trace.tolist() == ref.trace.tolist()
        assert r.stats["tests"] == ref.tests
    ha.free()
    hb.free()


def test_wait_times_out_on_a_running_mine_then_completes(dic):
    db = synth.planted_paper_scale(n=300_000)
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    ref = dic.mine(h, db.minsup, db.M).itemsets()
    # the ROWS path takes a while on this database: a 1 ms wait runs out
    job = dic.mine_async(h, db.minsup, db.M, path="rows")
    with pytest.raises(dic.DicError) as e:
        job.wait(timeout_ms=1)
    assert e.value.status == dic.dic.DIC_ETIMEOUT
    with pytest.raises(dic.DicError) as e2:
        h.free()                     # the database is busy while the job runs
    assert e2.value.status == dic.dic.DIC_EBUSY
    assert job.wait().itemsets() == ref
    h.free()


def test_async_argument_errors(dic):
    a = synth.planted_small()
    h = dic.load_db_csr(a.row_ptr, a.items, a.n, a.m)
    with pytest.raises(dic.DicError):
        dic.mine_async(h, 0, 10)
    with pytest.raises(dic.DicError):
        dic.mine_async(h, 10, 0)
    job = dic.mine_async(h, a.minsup, a.M)
    job.wait()
    with pytest.raises(dic.DicError):
        job.wait()                   # a job is waited once
    h.free()
