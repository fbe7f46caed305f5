"""Autotuner: choice, cache and the exactness check (CPU, with a stand-in
timing function), and on the GPU the tuned mine against the oracle."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1812_10959_gb300 import autotune  # noqa: E402


class _Db:
    n, m = 1000, 64


def test_picks_fastest_and_caches(tmp_path):
    calls = []

    def run(kw):
        calls.append(kw)
        sec = {"bitslice": 2.0, "tensor": 1.0, "auto": 3.0}[kw["path"]] + 0.01 * kw["tile_words"]
        return ("same",), sec

    path = str(tmp_path / "tune.json")
    t = autotune.Tuner(cache_path=path, run=run)
    c = t.tune(_Db(), 10, 100)
    assert (c.path, c.tile_words) == ("tensor", 8)
    assert len(calls) == len(autotune.CANDIDATES)
    # a second tuner reads the persisted choice and times nothing
    calls.clear()
    t2 = autotune.Tuner(cache_path=path, run=run)
    c2 = t2.tune(_Db(), 10, 100)
    assert (c2.path, c2.tile_words, c2.count_form) == (c.path, c.tile_words, c.count_form)
    assert calls == []
    # another shape is tuned afresh
    t2.tune(_Db(), 11, 100)
    assert len(calls) == len(autotune.CANDIDATES)


def test_result_change_is_an_error():
    n = [0]

    def run(kw):
        n[0] += 1
        return (("a",) if n[0] == 1 else ("b",)), 1.0

    with pytest.raises(RuntimeError):
        autotune.Tuner(run=run).tune(_Db(), 5, 50)


@pytest.mark.gpu
def test_tuned_mine_equals_oracle(tmp_path):
    import oracle
    import synth
    from paper_1812_10959_gb300 import dic
    db = synth.planted_small(3)
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    t = autotune.Tuner(cache_path=str(tmp_path / "t.json"), repeats=1)
    res = t.mine(h, db.minsup, db.M)
    ref = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M)
    assert res.itemsets() == ref.itemsets
    assert np.array_equal(res.trace, ref.trace)
    choice = t.tune(h, db.minsup, db.M)
    assert len(choice.timings) == len(autotune.CANDIDATES)
    h.free()


@pytest.mark.gpu
def test_invalid_options_rejected():
    import synth
    from paper_1812_10959_gb300 import dic
    db = synth.planted_small(0)
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    with pytest.raises(dic.DicError):
        dic.mine(h, db.minsup, db.M, tile_words=12)
    h.free()
