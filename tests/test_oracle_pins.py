"""Pins for the CPU oracle against facts that do not come from the oracle
itself: brute-force enumeration, closed forms, a textbook miner (Apriori,
Section 3), numpy's bit packing, and hand-worked runs of Algorithms 2-5."""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth
from golden_io import hand_examples, to_csr


def rand_db(rng, n, m, p):
    rows = [sorted(np.flatnonzero(rng.random(m) < p).tolist()) for _ in range(n)]
    rp, it = to_csr(rows)
    return rows, rp, it


def brute_python(rows, m, minsup):
    """Problem statement of Section 1 written out: every non-empty subset."""
    out = []
    sets = [set(r) for r in rows]
    for k in range(1, m + 1):
        for X in itertools.combinations(range(m), k):
            s = sum(1 for T in sets if set(X) <= T)
            if s >= minsup:
                out.append((X, s))
    return out


# ---------------------------------------------------------------- packing
@pytest.mark.parametrize("m", [1, 5, 63, 64, 65, 100, 130, 257])
def test_pack_matches_numpy_packbits(m):
    rng = np.random.default_rng(m)
    rows, rp, it = rand_db(rng, 37, m, 0.3)
    dense = np.zeros((37, m), dtype=np.uint8)
    for t, r in enumerate(rows):
        dense[t, r] = 1
    W = (m + 63) // 64
    padded = np.zeros((37, W * 64), dtype=np.uint8)
    padded[:, :m] = dense
    ref = np.packbits(padded, axis=1, bitorder="little").view("<u8").reshape(37, W)
    assert np.array_equal(oracle.pack(rp, it, 37, m), ref)


# ---------------------------------------------------- brute force / support
def test_bruteforce_matches_definition():
    rng = np.random.default_rng(1)
    for trial in range(6):
        m = int(rng.integers(1, 8))
        n = int(rng.integers(0, 25))
        rows, rp, it = rand_db(rng, n, m, 0.5)
        for minsup in (1, 2, 5):
            got = oracle.bruteforce(rp, it, n, m, minsup).itemsets
            assert got == brute_python(rows, m, minsup)


def test_support_and_pairs_match_definition():
    rng = np.random.default_rng(2)
    rows, rp, it = rand_db(rng, 60, 9, 0.4)
    sets = [set(r) for r in rows]
    qs = [c for k in (1, 2, 3) for c in itertools.combinations(range(9), k)]
    got = oracle.support(rp, it, 60, 9, qs)
    assert [int(x) for x in got] == [sum(1 for T in sets if set(q) <= T) for q in qs]
    P = oracle.pair_supports(rp, it, 60, 9)
    for a in range(9):
        for b in range(9):
            assert P[a, b] == sum(1 for T in sets if a in T and b in T)


# ------------------------------------------------- DIC vs brute force
@pytest.mark.parametrize("seed", range(8))
def test_dic_matches_bruteforce_every_M(seed):
    rng = np.random.default_rng(100 + seed)
    m = int(rng.integers(1, 13))
    n = int(rng.integers(1, 200))
    rows, rp, it = rand_db(rng, n, m, float(rng.uniform(0.2, 0.7)))
    for minsup in sorted({1, 2, max(1, n // 10), max(1, n // 3), n}):
        ref = oracle.bruteforce(rp, it, n, m, minsup).itemsets
        for M in sorted({1, 2, 7, math.ceil(n / 3), n, n + 5}):
            r = oracle.dic(rp, it, n, m, minsup, M)
            assert r.itemsets == ref, (n, m, minsup, M)
            assert r.violations == 0
            rc = oracle.dic_classic(rp, it, n, m, minsup, M)
            assert rc.itemsets == ref
            assert rc.violations == 0


def test_dic_wide_items_cross_word():
    """Items on both sides of 64-bit word boundaries (m = 130)."""
    rng = np.random.default_rng(7)
    m, n = 130, 300
    base = [0, 63, 64, 65, 127, 128, 129]
    rows = []
    for _ in range(n):
        r = [x for x in base if rng.random() < 0.6] + list(rng.integers(0, m, 3))
        rows.append(sorted(set(int(x) for x in r)))
    rp, it = to_csr(rows)
    ap = oracle.apriori(rp, it, n, m, 30).itemsets
    for M in (1, 17, 100, 300):
        assert oracle.dic(rp, it, n, m, 30, M).itemsets == ap
    assert any(len(s) >= 4 for s, _ in ap)


def test_dic_matches_apriori_planted_small():
    db = synth.planted_small()
    ap = oracle.apriori(db.row_ptr, db.items, db.n, db.m, db.minsup)
    r = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M)
    assert r.itemsets == ap.itemsets
    assert r.violations == 0
    assert len(r.itemsets) > 500 and max(len(s) for s, _ in r.itemsets) >= 3


# ------------------------------------------------------------ closed forms
def test_closed_form_minsup_n_is_powerset_of_intersection():
    rng = np.random.default_rng(3)
    m, n = 12, 40
    core = [1, 4, 5, 9]
    rows = [sorted(set(core + [int(x) for x in np.flatnonzero(rng.random(m) < 0.3)])) for _ in range(n)]
    inter = sorted(set.intersection(*[set(r) for r in rows]))
    rp, it = to_csr(rows)
    r = oracle.dic(rp, it, n, m, n, 7)
    exp = [(X, n) for k in range(1, len(inter) + 1) for X in itertools.combinations(inter, k)]
    assert r.itemsets == exp
    assert len(r.itemsets) == 2 ** len(inter) - 1


def test_closed_form_single_and_repeated_rows():
    T = [0, 3, 7, 8, 11]
    for reps in (1, 5):
        rows = [T] * reps
        rp, it = to_csr(rows)
        r = oracle.dic(rp, it, reps, 12, reps, 1)
        exp = [(X, reps) for k in range(1, 6) for X in itertools.combinations(T, k)]
        assert r.itemsets == exp


def test_closed_form_disjoint_blocks():
    blocks = [[0, 1, 2], [5, 6], [9, 10, 11, 12]]
    rows = [b for b in blocks for _ in range(4)]
    rp, it = to_csr(rows)
    r = oracle.dic(rp, it, len(rows), 13, 4, 3)
    exp = sorted([(X, 4) for b in blocks for k in range(1, len(b) + 1)
                  for X in itertools.combinations(b, k)], key=lambda p: (len(p[0]), p[0]))
    assert r.itemsets == exp


def test_empty_database_and_empty_rows():
    rp, it = to_csr([])
    assert oracle.dic(rp, it, 0, 5, 1, 3).itemsets == []
    rp, it = to_csr([[], [], [2], []])
    assert oracle.dic(rp, it, 4, 5, 1, 3).itemsets == [((2,), 1)]
    with pytest.raises(ValueError):
        oracle.dic(rp, it, 4, 5, 0, 3)
    with pytest.raises(ValueError):
        oracle.dic(rp, it, 4, 5, 1, 0)


# ------------------------------------------- M = n reduces to Apriori levels
def test_M_equals_n_is_apriori_level_by_level():
    db = synth.planted_small()
    r = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.n)
    ap = oracle.apriori(db.row_ptr, db.items, db.n, db.m, db.minsup)
    assert r.itemsets == ap.itemsets
    # one stop per level: the dashed count is |C_k|, promotions are |L_k|
    assert np.array_equal(r.trace[:, 4], ap.trace[:, 4][:len(r.trace)])
    assert np.array_equal(r.trace[:, 5], ap.trace[:, 5][:len(r.trace)])
    assert (r.trace[:, 1] == 1).all()


# ------------------------------------------------------------- invariants
def test_invariants_test_count_and_antimonotone():
    db = synth.planted_small()
    for M in (333, 1000, 4000):
        r = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, M)
        tr = r.trace.astype(np.int64)
        assert r.tests == db.m * db.n + int((tr[:, 4] * (tr[:, 3] - tr[:, 2])).sum())
        # every generated candidate is solidified or pruned, never lost
        gen = int(tr[:, 7].sum()) + (lambda L1: L1 * (L1 - 1) // 2)(
            sum(1 for s, _ in r.itemsets if len(s) == 1))
        assert gen == int(tr[:, 6].sum() + tr[:, 8].sum())
        d = r.as_dict()
        for X, s in d.items():
            for j in range(len(X)):
                sub = X[:j] + X[j + 1:]
                if sub:
                    assert sub in d and d[sub] >= s  # downward closed, anti-monotone


# ------------------------------------------------------ hand-worked runs
@pytest.mark.parametrize("ex", hand_examples(), ids=lambda e: e["name"])
def test_hand_worked_examples(ex):
    rp, it = to_csr(ex["rows"])
    r = oracle.dic(rp, it, ex["n"], ex["m"], ex["minsup"], ex["M"])
    assert r.itemsets == ex["L"]
    assert r.trace.tolist() == ex["trace"]
    assert r.tests == ex["tests"]
    assert oracle.bruteforce(rp, it, ex["n"], ex["m"], ex["minsup"]).itemsets == ex["L"]


# ---------------------------------------------------------------- rules
def _rules_direct(rows, m, minsup, num, den):
    """Every split X -> Y (disjoint, non-empty) of a frequent X | Y, with
    supports counted by scanning the rows and confidence compared as
    fractions: an enumeration independent of the oracle's."""
    from fractions import Fraction
    sets = [frozenset(r) for r in rows]

    def supp(s):
        return sum(1 for t in sets if s <= t)

    out = []
    for zmask in range(1, 1 << m):
        z = [i for i in range(m) if zmask >> i & 1]
        if len(z) < 2:
            continue
        sz = supp(frozenset(z))
        if sz < minsup:
            continue
        for xmask in range(1, 1 << m):
            if xmask & ~zmask or xmask == zmask:
                continue
            x = tuple(i for i in range(m) if xmask >> i & 1)
            y = tuple(i for i in z if not xmask >> i & 1)
            sx = supp(frozenset(x))
            if Fraction(sz, sx) >= Fraction(num, den):
                out.append((x, y, sz, sx))
    out.sort(key=lambda r: (len(r[0]), r[0], len(r[1]), r[1]))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_rules_match_direct_enumeration(seed):
    rng = np.random.default_rng(4000 + seed)
    m = int(rng.integers(2, 9))
    n = int(rng.integers(1, 50))
    rows = [np.flatnonzero(rng.random(m) < 0.5).tolist() for _ in range(n)]
    rp, it = to_csr(rows)
    minsup = max(1, n // 6)
    L = oracle.bruteforce(rp, it, n, m, minsup).itemsets
    for num, den in ((0, 1), (1, 2), (2, 3), (1, 1)):
        assert oracle.rules(L, num, den) == _rules_direct(rows, m, minsup, num, den)


def test_rules_closed_form_identical_rows():
    # r copies of one row T, minsup 1: every split of every subset holds at
    # confidence 1; there are 3^k - 2^(k+1) + 1 of them
    k, r = 6, 4
    rows = [list(range(k))] * r
    rp, it = to_csr(rows)
    L = oracle.bruteforce(rp, it, r, k, 1).itemsets
    got = oracle.rules(L, 1, 1)
    assert len(got) == 3 ** k - 2 ** (k + 1) + 1
    assert all(sz == r and sx == r for _, _, sz, sx in got)
