"""Failure detection in the forms that fault no GPU: errors made on the host.

* An allocation that fails part-way through a mine (injected on the host at
  every allocation the mine makes) gives DIC_ENOMEM, the call releases every
  working buffer it took (the memory pool's bytes in use return to where they
  were), and the next mine on the same process is exact.
* A wait with a short limit on a query still running in the request server
  gives DIC_ETIMEOUT, and the ticket can be waited again for its result.
"""
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dic():
    import paper_1812_10959_gb300 as d
    return d


@pytest.mark.parametrize("path", ["auto", "tensor", "rows"])
def test_allocation_failure_at_every_point_releases_everything(dic, path):
    import torch
    rp, it = synth.planted(seed=5, n=3000, m=70, n_patterns=60, pat_len_mean=4.0,
                           tx_len_mean=9.0)
    n, m, minsup, M = 3000, 70, 60, 700
    ref = oracle.dic(rp, it, n, m, minsup, M)
    h = dic.load_db_csr(rp, it, n, m)
    dic.mine(h, minsup, M, path=path)          # warm the pool
    torch.cuda.synchronize()
    base = dic.dic.debug_pool_used()
    failures = 0
    for after in range(400):
        dic.dic.debug_fail_device_alloc(after)
        try:
            r = dic.mine(h, minsup, M, path=path)
        except dic.DicError as e:
            assert e.status == dic.dic.DIC_ENOMEM, str(e)
            assert "injected" in str(e)
            failures += 1
            torch.cuda.synchronize()
            assert dic.dic.debug_pool_used() == base
            continue
        # `after` is past the mine's last allocation: the hook did not fire
        dic.dic.debug_fail_device_alloc(-1)
        assert r.itemsets() == ref.itemsets
        assert r.trace.tolist() == ref.trace.tolist()
        break
    else:
        pytest.fail("the mine allocated more than 400 buffers")
    assert failures >= 10
    torch.cuda.synchronize()
    assert dic.dic.debug_pool_used() == base
    h.free()


def test_server_wait_times_out_on_a_running_query_and_can_wait_again(dic):
    db = synth.planted_paper_scale(n=300_000)
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    alone = dic.mine(h, db.minsup, db.M)
    srv = dic.Server(max_slots=4, path="rows")
    t = srv.submit(h, db.minsup, db.M)
    with pytest.raises(dic.DicError) as e:
        srv.wait(t, timeout_ms=1)
    assert e.value.status == dic.dic.DIC_ETIMEOUT
    got = srv.wait(t)
    assert got.itemsets() == alone.itemsets()
    srv.close()
    h.free()
