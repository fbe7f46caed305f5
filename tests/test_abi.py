"""The C-ABI library loads on a machine without a GPU, exports every entry
point include/dic.h declares, and rejects bad arguments before any device
work."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dic.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \*]*?\b(dic_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1812_10959_gb300 import build as pb
    return pb.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dic_load_db", "dic_load_db_csr", "dic_load_db_device", "dic_mine",
                 "dic_mine_ex", "dic_mine_async", "dic_mine_wait", "dic_mine_batch",
                 "dic_result_copy", "dic_result_trace",
                 "dic_db_free", "dic_result_free", "dic_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (dic_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for f in declared_functions():
        assert getattr(lib, f) is not None


def test_host_side_validation_without_gpu(libpath):
    import paper_1812_10959_gb300 as dic
    lib = dic.dic.lib()
    assert lib.dic_abi_version() == 1
    assert lib.dic_minsup_count(10_000, 0.02) == 200
    assert lib.dic_minsup_count(1_000_000, 0.0025) == 2500
    assert lib.dic_minsup_count(7, 0.0) == 1
    assert lib.dic_status_str(4) == b"capacity exceeded"
    # padding bits beyond m are rejected on the host, before any CUDA call
    words = np.array([[1 << 5]], dtype=np.uint64)
    with pytest.raises(dic.DicError) as e:
        dic.load_db(words, 1, 5)
    assert e.value.status == dic.dic.DIC_EINVAL
    with pytest.raises(dic.DicError) as e:
        dic.load_db(words, 1, 0)
    assert e.value.status == dic.dic.DIC_EINVAL
    # row_ptr must start at 0 and not decrease
    with pytest.raises(dic.DicError):
        dic.load_db_csr(np.array([1, 2], dtype=np.uint64), np.array([0], dtype=np.uint32), 1, 4)
    with pytest.raises(dic.DicError):
        dic.load_db_csr(np.array([0, 2, 1], dtype=np.uint64), np.array([0, 1], dtype=np.uint32),
                        2, 4)
    # n >= 2^31 is refused
    h = ctypes.c_void_p()
    assert lib.dic_load_db(None, 1 << 31, 4, ctypes.byref(h)) == dic.dic.DIC_EINVAL
    # mining arguments
    assert lib.dic_mine(None, 1, 1, ctypes.byref(h)) == dic.dic.DIC_EINVAL


def test_options_defaults_and_rules_validation_without_gpu(libpath):
    import paper_1812_10959_gb300 as dic
    d = dic.dic
    o = d.Options()
    d.lib().dic_options_init(ctypes.byref(o))
    assert o.struct_size == ctypes.sizeof(d.Options)
    assert (o.count_path, o.use_graph, o.profile, o.tile_words, o.count_form, o.algorithm) == \
        (0, 1, 0, 0, 0, 0)
    # the rules entry point checks its arguments on the host, before any CUDA call
    W = 1
    masks = np.array([[0b11]], dtype=np.uint64)
    res = d.Result(W, masks, np.array([3], dtype=np.uint32), np.array([5], dtype=np.uint32),
                   np.zeros((0, 9), dtype=np.uint64), {})
    with pytest.raises(d.DicError) as e:
        d.rules(res, 1, 2, m=2)            # size 3 is not the popcount 2
    assert e.value.status == d.DIC_EINVAL
    with pytest.raises(d.DicError) as e:
        d.rules(res, 1, 0, m=2)            # zero denominator
    assert e.value.status == d.DIC_EINVAL
    wide = d.Result(W, np.array([[1 << 40]], dtype=np.uint64), np.array([1], dtype=np.uint32),
                    np.array([5], dtype=np.uint32), np.zeros((0, 9), dtype=np.uint64), {})
    with pytest.raises(d.DicError) as e:
        d.rules(wide, 1, 2, m=10)          # item 40 >= m
    assert e.value.status == d.DIC_EINVAL
    big = d.Result(W, np.array([[(1 << 32) - 1]], dtype=np.uint64),
                   np.array([32], dtype=np.uint32), np.array([5], dtype=np.uint32),
                   np.zeros((0, 9), dtype=np.uint64), {})
    with pytest.raises(d.DicError) as e:
        d.rules(big, 1, 2, m=64)           # more than 31 items in one itemset
    assert e.value.status == d.DIC_ECAPACITY
    # no itemset of two or more items: no rules and no device work
    single = d.Result(W, np.array([[1], [2]], dtype=np.uint64), np.array([1, 1], dtype=np.uint32),
                      np.array([5, 4], dtype=np.uint32), np.zeros((0, 9), dtype=np.uint64), {})
    assert d.rules(single, 1, 2, m=2) == []
