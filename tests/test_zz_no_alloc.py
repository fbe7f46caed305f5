"""dic_count_support_noalloc, the entry point for callers that cannot
allocate device memory (fixed memory budgets, runtimes that own all device
memory): through the C ABI, its counts must equal the supports that
dic_mine reports for the same itemsets, on two calls in a row (the second
call reuses the scratch array the first one left behind). Runs last so that a
failure here never hides the result of another test."""
import ctypes

import numpy as np
import pytest

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
    small = synth.planted_small()
    rng = np.random.default_rng(31)
    rows = []
    for _ in range(5000):
        r = [x for x in (0, 63, 64, 65, 127, 128, 129) if rng.random() < 0.5]
        rows.append(r + rng.integers(0, 130, 6).tolist())
    rp, it = to_csr(rows)
    return [(small.row_ptr, small.items, small.n, small.m, small.minsup, small.M),
            (rp, it, 5000, 130, 400, 700)]


def test_noalloc_counts_match_dic_mine_on_two_calls():
    import torch
    import paper_1812_10959_gb300 as dic
    lib = dic.dic.lib()
    stream = torch.cuda.Stream()
    for rp, it, n, m, minsup, M in _databases():
        db = dic.load_db_csr(rp, it, n, m)
        res = dic.mine(db, minsup, M)
        assert len(res.k) > 50
        masks = torch.from_numpy(res.masks.view(np.int64).copy()).cuda()
        supp = torch.full((len(res.k),), -1, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        assert _noalloc(lib, db, masks, supp, stream) == dic.dic.DIC_OK
        stream.synchronize()
        got = supp.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, res.support)
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
