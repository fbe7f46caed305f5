"""Negative-border certificate of a mining result (test infrastructure).

A set L of (itemset, support) pairs is exactly the answer of the problem in
Section 1 -- every non-empty itemset X with supp(X) >= minsup, with its exact
support -- iff all of the following hold:

  (i)   every reported support equals the support counted directly from the
        rows, and is >= minsup;
  (ii)  L is downward closed (every non-empty subset of a member is a
        member; anti-monotonicity of support makes this necessary);
  (iii) every itemset of the negative border -- an itemset not in L whose
        subsets with one item fewer are all in L, single items included --
        has support < minsup.

(If some frequent X were missing, a minimal missing one would lie on the
border and violate (iii).) The checks below need no second miner, so they
run at sizes the serial oracle cannot mine in a test: single items by
``np.bincount``, every pair among the frequent items at once (the whole pair
border) by ``oracle.pair_supports`` or, for long rows, a dense 0/1
matrix product (integer-valued float32 sums below 2^24 are exact), and every
larger itemset and larger border candidate by ``oracle.support`` (tid-list
intersection).
"""
from __future__ import annotations

import numpy as np

import oracle


def item_counts(row_ptr, items, m):
    return np.bincount(np.asarray(items, dtype=np.int64), minlength=m)[:m]


def pair_matrix(row_ptr, items, n, m, cols, dense=None):
    """uint64 [len(cols), len(cols)]: rows containing both cols[a] and
    cols[b] (diagonal: rows containing cols[a]). `dense` forces the method
    (None: by the work of the sparse count)."""
    cols = np.asarray(cols, dtype=np.int64)
    lens = np.diff(np.asarray(row_ptr, dtype=np.int64))
    work_sparse = float((lens.astype(np.float64) ** 2).sum())
    if dense is False or (dense is None and work_sparse <= 2e9):
        P = oracle.pair_supports(row_ptr, items, n, m)
        return P[np.ix_(cols, cols)].astype(np.uint64)
    # long rows: dense 0/1 rows restricted to `cols`, X^T X in row chunks
    # (each chunk's counts are integers below 2^24, exact in float32)
    pos = np.full(m, -1, dtype=np.int64)
    pos[cols] = np.arange(len(cols))
    rp = np.asarray(row_ptr, dtype=np.int64)
    it = np.asarray(items, dtype=np.int64)
    out = np.zeros((len(cols), len(cols)), dtype=np.uint64)
    chunk = 1 << 16
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        seg = it[rp[r0]:rp[r1]]
        rows = np.repeat(np.arange(r1 - r0), lens[r0:r1])
        keep = pos[seg] >= 0
        X = np.zeros((r1 - r0, len(cols)), dtype=np.float32)
        X[rows[keep], pos[seg[keep]]] = 1.0
        out += np.rint(X.T @ X).astype(np.uint64)
    return out


def border_candidates(level_sets, frequent):
    """Itemsets of size k+1 not in `frequent` whose k-subsets are all in it,
    built from the frequent k-itemsets `level_sets` (sorted tuples): joins
    of two members that share their first k-1 items."""
    by_prefix = {}
    for s in level_sets:
        by_prefix.setdefault(s[:-1], []).append(s[-1])
    out = []
    for pre, lasts in by_prefix.items():
        lasts = sorted(lasts)
        for i in range(len(lasts)):
            for j in range(i + 1, len(lasts)):
                c = pre + (lasts[i], lasts[j])
                if c in frequent:
                    continue
                if all(c[:q] + c[q + 1:] in frequent for q in range(len(c))):
                    out.append(c)
    return out


def certify(row_ptr, items, n, m, minsup, got, pairs=None):
    """Assert that `got` ([(items_tuple, support)], canonical order) is the
    exact frequent-itemset answer. `pairs` may hold a precomputed
    (cols, pair_matrix) for this database (reused across thresholds).
    Returns a dict of what was checked."""
    got = list(got)
    # canonical order: size, then lexicographic; no duplicates
    keys = [(len(s), s) for s, _ in got]
    assert keys == sorted(keys) and len(set(keys)) == len(keys), "order or duplicates"
    L = dict(got)
    for s, v in got:
        assert v >= minsup, f"{s} reported with support {v} < minsup"
        assert len(s) >= 1 and list(s) == sorted(set(s)) and s[-1] < m
    # (ii) downward closed
    for s, _ in got:
        if len(s) > 1:
            for q in range(len(s)):
                assert s[:q] + s[q + 1:] in L, f"{s} reported without its subset"
    # (i)+(iii) for single items: every item, frequent or not
    cnt = item_counts(row_ptr, items, m)
    exp1 = [((i,), int(cnt[i])) for i in range(m) if cnt[i] >= minsup]
    assert [x for x in got if len(x[0]) == 1] == exp1, "1-itemsets"
    l1 = [s[0] for s, _ in exp1]
    # (i)+(iii) for pairs: every pair of frequent items
    if pairs is not None and set(l1) <= set(pairs[0]):
        cols, P = pairs
        idx = {c: q for q, c in enumerate(cols)}
        sub = np.asarray([idx[c] for c in l1], dtype=np.int64)
        P = P[np.ix_(sub, sub)]
    else:
        P = pair_matrix(row_ptr, items, n, m, l1)
    ia, ib = np.nonzero(np.triu(P, 1) >= minsup)
    exp2 = sorted(((l1[a], l1[b]), int(P[a, b])) for a, b in zip(ia, ib))
    assert [x for x in got if len(x[0]) == 2] == exp2, "2-itemsets (whole pair border)"
    n_pair_border = len(l1) * (len(l1) - 1) // 2 - len(exp2)
    # (i) for larger itemsets, (iii) for larger border candidates
    big = [s for s, _ in got if len(s) >= 3]
    n_border, k = 0, 2
    frequent = set(L)
    while True:
        level = sorted(s for s in frequent if len(s) == k)
        cand = border_candidates(level, frequent)
        if cand:
            sup = oracle.support(row_ptr, items, n, m, cand)
            bad = [c for c, v in zip(cand, sup) if v >= minsup]
            assert not bad, f"frequent itemsets missing from the result: {bad[:5]}"
        n_border += len(cand)
        if not level:
            break
        k += 1
    if big:
        sup = oracle.support(row_ptr, items, n, m, big)
        assert [int(v) for v in sup] == [L[s] for s in big], "supports of itemsets of size >= 3"
    return {"itemsets": len(got), "l1": len(l1), "pairs": len(exp2),
            "pair_border": n_pair_border, "larger": len(big), "larger_border": n_border,
            "item_border": m - len(l1)}
