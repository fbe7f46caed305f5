"""CPU pins of the negative-border certificate used by the full-size GPU
parity tests: it accepts the brute-force answer and rejects answers with one
planted mistake of each kind (a missing itemset, a wrong support, an extra
infrequent itemset, a missing subset); its two pair counters agree."""
import numpy as np
import pytest

import oracle
import synth
from certificate import certify, pair_matrix
from golden_io import to_csr


def small_db(seed, n=120, m=12, p=0.35):
    rng = np.random.default_rng(seed)
    rows = [np.flatnonzero(rng.random(m) < p).tolist() for _ in range(n)]
    rows += [[1, 2, 3, 4]] * 20          # a planted 4-itemset
    rp, it = to_csr(rows)
    return rp, it, len(rows), m


@pytest.mark.parametrize("seed", range(4))
def test_accepts_the_bruteforce_answer(seed):
    rp, it, n, m = small_db(seed)
    for minsup in (8, 20, 30):
        ref = oracle.bruteforce(rp, it, n, m, minsup).itemsets
        info = certify(rp, it, n, m, minsup, ref)
        assert info["itemsets"] == len(ref)


def mutations(ref, minsup, rp, it, n, m):
    """One planted mistake per mutant (each still sorted canonically)."""
    key = lambda x: (len(x[0]), x[0])
    L = dict(ref)
    big = [s for s, _ in ref if len(s) >= 2]
    maximal = [s for s in big if not any(set(s) < set(t) for t in L)]
    out = []
    # a maximal itemset dropped: still downward closed, caught by the border
    out.append([x for x in ref if x[0] != maximal[0]])
    # a non-maximal one dropped: caught by closure (or the pair/border check)
    nonmax = [s for s in big if s not in maximal]
    if nonmax:
        out.append([x for x in ref if x[0] != nonmax[0]])
    # a support off by one, at each size
    for k in sorted({len(s) for s, _ in ref}):
        s = next(x for x in ref if len(x[0]) == k)
        out.append(sorted([(x[0], x[1] + (1 if x[0] == s[0] else 0)) for x in ref], key=key))
    # an infrequent itemset whose subsets are all frequent, with its true support
    freq = set(L)
    for a in range(m):
        for b in range(a + 1, m):
            if (a,) in freq and (b,) in freq and (a, b) not in freq:
                v = int(oracle.support(rp, it, n, m, [(a, b)])[0])
                out.append(sorted(ref + [((a, b), v)], key=key))
                return out
    return out


@pytest.mark.parametrize("seed", range(4))
def test_rejects_every_planted_mistake(seed):
    rp, it, n, m = small_db(seed)
    minsup = 20
    ref = oracle.bruteforce(rp, it, n, m, minsup).itemsets
    muts = mutations(ref, minsup, rp, it, n, m)
    assert len(muts) >= 4
    for bad in muts:
        with pytest.raises(AssertionError):
            certify(rp, it, n, m, minsup, bad)


def test_sparse_and_dense_pair_counts_agree():
    rp, it = synth.planted(seed=3, n=3000, m=150, n_patterns=60, pat_len_mean=5.0,
                           tx_len_mean=25.0)
    cols = list(range(0, 150, 2))
    a = pair_matrix(rp, it, 3000, 150, cols, dense=False)
    b = pair_matrix(rp, it, 3000, 150, cols, dense=True)
    assert np.array_equal(a, b)
    d = synth.Database("x", 3000, 150, rp, it, 1, 1).dense()
    assert np.array_equal(a, (d[:, cols].T.astype(np.int64) @ d[:, cols]).astype(np.uint64))


def test_certifies_the_oracle_on_the_planted_small_workload():
    db = synth.planted_small()
    ref = oracle.dic(db.row_ptr, db.items, db.n, db.m, db.minsup, db.M).itemsets
    info = certify(db.row_ptr, db.items, db.n, db.m, db.minsup, ref)
    assert info["larger"] > 0 and info["larger_border"] > 0 and info["pair_border"] > 0
