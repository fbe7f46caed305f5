"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle:
itemsets, integer supports, the per-stop trace and the test count."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from golden_io import hand_examples, to_csr
from gpu_util import packbits_rows

pytestmark = pytest.mark.gpu
PATHS = ["rows", "bitslice", "tensor", "auto"]


@pytest.fixture(scope="module")
def dic():
    import torch
    assert torch.cuda.is_available()
    import paper_1812_10959_gb300 as d
    return d


def check(dic, rp, it, n, m, minsup, M, path, trace=True):
    db = dic.load_db_csr(rp, it, n, m)
    res = dic.mine(db, minsup, M, path=path)
    ref = oracle.dic(rp, it, n, m, minsup, M)
    assert res.itemsets() == ref.itemsets
    if trace:
        assert res.trace.tolist() == ref.trace.tolist()
        assert res.stats["tests"] == ref.tests
    db.free()
    return res, ref


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("ex", hand_examples(), ids=lambda e: e["name"])
def test_hand_worked_examples(dic, ex, path):
    rp, it = to_csr(ex["rows"])
    res, _ = check(dic, rp, it, ex["n"], ex["m"], ex["minsup"], ex["M"], path)
    assert res.itemsets() == ex["L"]
    assert res.trace.tolist() == ex["trace"]
    assert res.stats["tests"] == ex["tests"]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("seed", range(10))
def test_random_small_every_M(dic, seed, path):
    rng = np.random.default_rng(500 + seed)
    m = int(rng.integers(1, 140))
    n = int(rng.integers(1, 400))
    p = float(rng.uniform(0.05, 0.5)) if m < 40 else float(rng.uniform(0.02, 0.1))
    rows = [np.flatnonzero(rng.random(m) < p).tolist() for _ in range(n)]
    rp, it = to_csr(rows)
    for minsup in sorted({1 if m <= 16 else max(2, n // 20), max(1, n // 8), n}):
        for M in sorted({1, 3, math.ceil(n / 3), n, n + 7}):
            check(dic, rp, it, n, m, minsup, M, path)


@pytest.mark.parametrize("path", PATHS)
def test_planted_small_full_size(dic, path):
    db = synth.planted_small()
    res, ref = check(dic, db.row_ptr, db.items, db.n, db.m, db.minsup, db.M, path)
    assert len(res.itemsets()) == 655


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("m", [64, 65, 130, 1000, 4096])
def test_word_boundaries_and_wide_rows(dic, m, path):
    """Planted patterns over items placed at 64-bit word edges; many words."""
    rng = np.random.default_rng(m)
    n = 1200
    edge = sorted({0, 62, 63, 64, 65, 127, 128, m - 1, m - 2} & set(range(m)))
    rows = []
    for _ in range(n):
        r = [x for x in edge if rng.random() < 0.55]
        r += rng.integers(0, m, 4).tolist()
        rows.append(r)
    rp, it = to_csr(rows)
    check(dic, rp, it, n, m, 150, 97, path)


def test_load_paths_agree(dic):
    import torch
    db = synth.planted_small()
    words = packbits_rows(db.row_ptr, db.items, db.n, db.m)
    a = dic.load_db(words, db.n, db.m)
    b = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    t = torch.from_numpy(words.view(np.int64)).cuda()
    c = dic.load_db_device(t, db.n, db.m)
    ra, rb, rc = (dic.mine(x, db.minsup, db.M).itemsets() for x in (a, b, c))
    assert ra == rb == rc
    for x in (a, b, c):
        x.free()


def test_edge_cases(dic):
    # n = 0
    rp, it = to_csr([])
    db = dic.load_db_csr(rp, it, 0, 8)
    r = dic.mine(db, 1, 5)
    assert r.itemsets() == [] and len(r.trace) == 0
    db.free()
    # empty rows, a single frequent item (no pairs), minsup above n
    rp, it = to_csr([[], [3], [], [3, 5]])
    db = dic.load_db_csr(rp, it, 4, 8)
    assert dic.mine(db, 2, 2).itemsets() == [((3,), 2)]
    assert dic.mine(db, 5, 2).itemsets() == []
    assert dic.mine(db, 1, 100).itemsets() == oracle.dic(rp, it, 4, 8, 1, 100).itemsets
    with pytest.raises(dic.DicError):
        dic.mine(db, 0, 2)
    with pytest.raises(dic.DicError):
        dic.mine(db, 1, 0)
    db.free()
    # an item id >= m is refused by the device packer
    with pytest.raises(dic.DicError):
        dic.load_db_csr(np.array([0, 1], dtype=np.uint64), np.array([9], dtype=np.uint32), 1, 8)
    # padding bits in device words are refused
    import torch
    t = torch.tensor([[1 << 9]], dtype=torch.int64, device="cuda")
    with pytest.raises(dic.DicError):
        dic.load_db_device(t, 1, 8)


@pytest.mark.parametrize("path", PATHS)
def test_growth_of_every_buffer(dic, path):
    """minsup = n over rows sharing 15 items: all 2^15-1 subsets are frequent,
    so the box set, the candidate store and the kernel width all grow."""
    core = list(range(3, 18))
    rng = np.random.default_rng(9)
    rows = [core + rng.integers(20, 60, 3).tolist() for _ in range(40)]
    rp, it = to_csr(rows)
    res, ref = check(dic, rp, it, 40, 60, 40, 7, path)
    assert len(res.itemsets()) >= 2 ** 15 - 1
    assert max(len(s) for s, _ in res.itemsets()) == 15


def test_capacity_limit_is_an_error_not_a_truncation(dic):
    core = list(range(10))
    rp, it = to_csr([core] * 5)
    db = dic.load_db_csr(rp, it, 5, 12)
    with pytest.raises(dic.DicError) as e:
        dic.mine(db, 5, 2, max_candidates=60)
    assert e.value.status == dic.dic.DIC_ECAPACITY
    assert len(dic.mine(db, 5, 2).itemsets()) == 2 ** 10 - 1
    db.free()


def test_repeatable_and_M_invariant(dic):
    db = synth.planted_small()
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    base = dic.mine(h, db.minsup, db.M).itemsets()
    for M in (1, 250, 999, 3333, 10_000, 20_000):
        assert dic.mine(h, db.minsup, M).itemsets() == base
    assert dic.mine(h, db.minsup, db.M).itemsets() == base
    h.free()


def test_paths_agree_on_wide_frequent_items(dic):
    """~1,600 frequent items out of 4,096 (the bitslice path then uses a
    narrower tile). All paths agree; the oracle pins the 1- and 2-itemsets
    exactly (pair co-occurrence counts, including the infrequent pairs) and
    the supports of every larger itemset."""
    rng = np.random.default_rng(77)
    n, m, minsup = 2000, 4096, 60
    hot = rng.choice(m, 1600, replace=False)
    pats = [rng.choice(hot, 5, replace=False) for _ in range(3)]
    rows = []
    for t in range(n):
        r = rng.choice(hot, 80, replace=False).tolist() + rng.integers(0, m, 5).tolist()
        for p in pats:
            if rng.random() < 0.06:
                r += p.tolist()
        rows.append(r)
    rp, it = to_csr(rows)
    db = dic.load_db_csr(rp, it, n, m)
    out = {path: dic.mine(db, minsup, 700, path=path)
           for path in ("rows", "bitslice", "tensor", "auto")}
    db.free()
    got = out["rows"].itemsets()
    assert got == out["bitslice"].itemsets() == out["tensor"].itemsets() == out["auto"].itemsets()
    assert out["tensor"].stats["path_launches"][3] > 0
    assert out["bitslice"].stats["l1"] > 1430
    assert out["bitslice"].stats["path_launches"][2] > 0
    P = oracle.pair_supports(rp, it, n, m)
    d = np.diag(P)
    exp1 = [((i,), int(d[i])) for i in range(m) if d[i] >= minsup]
    iu = np.argwhere(np.triu(P, 1) >= minsup)
    exp2 = sorted(((int(a), int(b)), int(P[a, b])) for a, b in iu)
    assert [x for x in got if len(x[0]) == 1] == exp1
    assert [x for x in got if len(x[0]) == 2] == exp2
    big = [x for x in got if len(x[0]) >= 3]
    assert big, "the planted patterns give itemsets of size >= 3"
    sup = oracle.support(rp, it, n, m, [s for s, _ in big])
    assert [int(v) for v in sup] == [v for _, v in big]
    gd = dict(got)
    for X, _ in big:
        for j in range(len(X)):
            assert X[:j] + X[j + 1:] in gd


@pytest.mark.parametrize("path", PATHS)
def test_growth_inside_the_first_group_of_stops(dic, path):
    """The candidate store overflows and the box set grows within the first
    stops enqueued together (and the window outgrows the first tile)."""
    rp, it = synth.planted(seed=5, n=3000, m=70, n_patterns=60, pat_len_mean=4.0,
                           tx_len_mean=9.0)
    res, ref = check(dic, rp, it, 3000, 70, 60, 700, path)
    assert len(res.itemsets()) == 1693


@pytest.fixture(scope="module")
def dense_small():
    return synth.dense_zipf(n=2000)


@pytest.mark.parametrize("path", PATHS)
def test_dense_reduced_rows_full_oracle(dic, dense_small, path):
    """Dense recipe (4,096 items, ~400 per row, minsup 20%) on 2,000 rows:
    exact itemsets and trace against the full oracle run."""
    db = dense_small
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    res = dic.mine(h, db.minsup, 400, path=path)
    h.free()
    ref = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, 400, superset_loop=False)
    assert res.itemsets() == ref.itemsets
    assert res.trace.tolist() == ref.trace.tolist()
    assert res.stats["tests"] == ref.tests
    assert res.stats["l1"] > 400


def test_dense_full_size(dic):
    """Dense recipe at its full size (200,000 rows), in the launch
    configuration bench.py uses: every 1-itemset exact, every reported
    itemset's support equal to the oracle's, the itemsets downward closed,
    and a seeded sample of the pair negative border infrequent; the ROWS path
    agrees."""
    db = synth.dense_zipf()
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    res = dic.mine(h, db.minsup, db.M, path="auto")
    got = res.itemsets()
    assert got == dic.mine(h, db.minsup, db.M, path="rows").itemsets()
    assert got == dic.mine(h, db.minsup, db.M, path="tensor").itemsets()
    h.free()
    freq = np.bincount(db.items, minlength=db.m)
    assert [x for x in got if len(x[0]) == 1] == [((i,), int(freq[i])) for i in range(db.m)
                                                  if freq[i] >= db.minsup]
    big = [x for x in got if len(x[0]) >= 2]
    assert len(big) > 100
    sup = oracle.support(db.row_ptr, db.items, db.n, db.m, [s for s, _ in big])
    assert [int(v) for v in sup] == [v for _, v in big]
    gd = dict(got)
    for X, _ in big:
        for j in range(len(X)):
            assert X[:j] + X[j + 1:] in gd
    l1 = [s[0] for s, _ in got if len(s) == 1]
    rng = np.random.default_rng(3)
    border = set()
    while len(border) < 3000:
        a, b = sorted(rng.choice(l1, 2, replace=False).tolist())
        if (a, b) not in gd:
            border.add((a, b))
    bs = oracle.support(db.row_ptr, db.items, db.n, db.m, sorted(border))
    assert (bs < db.minsup).all()


@pytest.mark.parametrize("path", PATHS)
def test_direct_launches_equal_graph_replays(dic, path):
    """Stops replayed as captured CUDA graphs and stops launched one kernel
    at a time give the same result and trace (and the oracle's)."""
    db = synth.planted_small()
    h = dic.load_db_csr(db.row_ptr, db.items, db.n, db.m)
    a = dic.mine(h, db.minsup, db.M, path=path, use_graph=True, profile=True)
    b = dic.mine(h, db.minsup, db.M, path=path, use_graph=False)
    h.free()
    ref = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M)
    assert a.itemsets() == b.itemsets() == ref.itemsets
    assert a.trace.tolist() == b.trace.tolist() == ref.trace.tolist()
    # one count launch per stop, or per iteration of the event-driven loop
    assert a.stats["count_launches"] >= (a.stats["event_iters"] if a.stats["event_loop"]
                                         else len(ref.trace))


def test_pair_gemm_split_over_few_large_blocks(dic):
    """Two blocks of 75,000 rows: the all-blocks pair GEMM has fewer (block,
    tile pair) CTAs than SMs, so each block's rows are split across CTAs
    whose 32-bit partial counts are added up. Result, trace and test count
    equal the oracle's."""
    n, m, minsup, M = 150_000, 300, 1_500, 75_000
    rp, it = synth.planted(5, n, m, 60, 4.0, 9.0)
    db = dic.load_db_csr(rp, it, n, m)
    r = dic.mine(db, minsup, M, path="tensor")
    db.free()
    ref = oracle.dic(rp, it, n, m, minsup, M, superset_loop=False)
    assert r.itemsets() == ref.itemsets
    assert r.trace.tolist() == ref.trace.tolist()
    assert r.stats["tests"] == ref.tests
