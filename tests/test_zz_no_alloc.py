"""dic_count_support_noalloc, the entry point for callers that cannot
allocate device memory (fixed memory budgets, runtimes that own all device
memory): through the C ABI, its counts must equal the supports that
dic_mine reports for the same itemsets and the oracle's tid-list supports,
on two calls in a row (the second call reuses the scratch array the first
one left behind). Databases taller than one slab of the scratch array
(65,536 rows up to 512 items; 8,192 rows at 4,096 items) cover the slab loop
and the accumulation of counts across slabs. Runs last so that a failure here
never hides the result of another test."""
import ctypes

import numpy as np
import pytest

import oracle
import synth
from golden_io import to_csr

pytestmark = pytest.mark.gpu


def _noalloc(lib, db, masks_dev, supp_dev, stream):
    lib.dic_count_support_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                              ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                              ctypes.c_void_p]
    lib.dic_count_support_noalloc.restype = ctypes.c_int
    return lib.dic_count_support_noalloc(db.device_words_ptr(), db.n, db.m, masks_dev.data_ptr(),
                                         masks_dev.shape[0], supp_dev.data_ptr(),
                                         stream.cuda_stream)


def _databases():
    """(row_ptr, items, n, m, minsup, M): one slab and several slabs."""
    small = synth.planted_small()
    rng = np.random.default_rng(31)
    rows = []
    for _ in range(5000):
        r = [x for x in (0, 63, 64, 65, 127, 128, 129) if rng.random() < 0.5]
        rows.append(r + rng.integers(0, 130, 6).tolist())
    rp, it = to_csr(rows)
    out = [(small.row_ptr, small.items, small.n, small.m, small.minsup, small.M),
           (rp, it, 5000, 130, 400, 700)]
    # three slabs of 65,536 rows (m = 100), the last one short
    rp, it = synth.planted(41, 150_000, 100, 200, 4.0, 10.0)
    out.append((rp, it, 150_000, 100, 3000, 15_000))
    # two slabs at m = 64 (one 64-bit word per row)
    rp, it = synth.planted(42, 70_001, 64, 128, 3.0, 4.0)
    out.append((rp, it, 70_001, 64, 1400, 7_000))
    # three slabs of 8,192 rows at the largest item count (4,096), ragged tail
    rp, it = synth.planted(43, 20_001, 4096, 400, 4.0, 30.0)
    out.append((rp, it, 20_001, 4096, 200, 2_000))
    return out


def _extra_itemsets(rng, m, frequent_items, count=64):
    """Itemsets of 1-4 items, mostly among frequent items (some with
    supports below minsup), plus the last item and word-edge items."""
    out = []
    pool = np.asarray(frequent_items if len(frequent_items) >= 4 else range(m))
    for q in range(count):
        k = 1 + q % 4
        s = rng.choice(pool, k, replace=False).tolist()
        if q % 7 == 0:
            s[0] = m - 1
        if q % 11 == 0 and m > 64:
            s[-1] = 63 + (q % 3)
        out.append(tuple(sorted(set(int(x) for x in s))))
    return out


def _masks(itemsets, m):
    W = (m + 63) // 64
    out = np.zeros((len(itemsets), W), dtype=np.uint64)
    for q, s in enumerate(itemsets):
        for x in s:
            out[q, x // 64] |= np.uint64(1) << np.uint64(x % 64)
    return out


def test_noalloc_counts_match_dic_mine_and_the_oracle_on_two_calls():
    import torch
    import paper_1812_10959_gb300 as dic
    lib = dic.dic.lib()
    stream = torch.cuda.Stream()
    rng = np.random.default_rng(5)
    for rp, it, n, m, minsup, M in _databases():
        db = dic.load_db_csr(rp, it, n, m)
        res = dic.mine(db, minsup, M)
        mined = [s for s, _ in res.itemsets()]
        assert len(mined) > 10
        freq1 = [s[0] for s in mined if len(s) == 1]
        extra = _extra_itemsets(rng, m, freq1)
        sets = mined + extra
        expect = oracle.support(rp, it, n, m, sets).astype(np.uint32)
        assert np.array_equal(expect[:len(mined)], res.support)
        masks = torch.from_numpy(_masks(sets, m).view(np.int64)).cuda()
        for call in range(2):
            supp = torch.full((len(sets),), -1 - call, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            assert _noalloc(lib, db, masks, supp, stream) == dic.dic.DIC_OK
            stream.synchronize()
            got = supp.cpu().numpy().view(np.uint32)
            assert np.array_equal(got[:len(mined)], res.support), (n, m, call)
            assert np.array_equal(got, expect), (n, m, call)
        db.free()


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch
    import paper_1812_10959_gb300 as dic
    lib = dic.dic.lib()
    n, m = 4, 5000
    words = torch.zeros((n, (m + 63) // 64), dtype=torch.int64, device="cuda")
    db = dic.load_db_device(words, n, m)
    masks = torch.zeros((1, (m + 63) // 64), dtype=torch.int64, device="cuda")
    supp = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = _noalloc(lib, db, masks, supp, torch.cuda.current_stream())
    assert rc == dic.dic.DIC_EINVAL
    assert b"4096" in lib.dic_last_error()
    db.free()
