// CPU oracle for Dynamic Itemset Counting (DIC) -- TEST INFRASTRUCTURE ONLY.
//
// This file is the plain, slow, serial statement of what the GPU path must
// compute. Only the tests, the smoke check and the benchmark's CPU-baseline
// leg load it; the CUDA library never does, and the two share no code.
//
// Contents (each follows the paper's text; all arithmetic is integer/exact):
//   oracle_pack        BitMask of every transaction, Section 4.1 (W words of
//                      64 bits, item p -> word p/64, bit p%64).
//   oracle_dic         ParallelDIC, Algorithm 2, run serially: FIRSTPASS
//                      (Section 4.2), COUNTSUPPORT (Algorithm 3), PRUNE
//                      (Algorithm 4), MAKECANDIDATES (Section 4.2 text plus
//                      the generation rule of Algorithm 1 / Section 3),
//                      CHECKFULLPASS (Algorithm 5). Emits L and a per-stop
//                      trace.
//   oracle_dic_classic The serial DIC of Algorithm 1: no first pass; every
//                      1-itemset starts as a dashed circle.
//   oracle_apriori     Level-wise Apriori, Section 3 (join + a-priori prune,
//                      count by item-list inclusion).
//   oracle_bruteforce  Every non-empty subset counted by sub-mask enumeration
//                      (problem statement, Section 1), m <= 24.
//   oracle_support     support(X) = |intersection of the items' tid-lists|.
//   oracle_pair_supports  co-occurrence count of every item pair.
//
// Readings of the paper taken here (the paper is silent or garbled there):
//   * minsup is an integer count; frequent means supp >= minsup.
//   * stop_max = ceil(n/M); block s is [(s-1)M, min(sM, n)); the prune bound
//     keeps the literal supp + M*(stop_max - stop) in 64-bit arithmetic.
//   * MAKECANDIDATES after PRUNE at a stop adds every C with |C| >= 3 whose
//     (|C|-1)-subsets are all boxes and at least one of them was promoted at
//     this stop; 2-itemset candidates come only from the first pass.
//   * Phase order within a stop: COUNT, PRUNE, MAKECANDIDATES, CHECKFULLPASS.
//     CHECKFULLPASS scans all of DASHED.
//   * The superset loop of PRUNE is run as written; it can only ever match the
//     pruned itemset itself (every subset of a lattice member is a box), and
//     a match on any other itemset is counted as a violation.
//   * A candidate generated twice is counted as a violation.
//   * Output L: SOLID boxes, 1-itemsets included, ordered by size then
//     lexicographically by ascending item ids.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <vector>

namespace {

typedef std::vector<uint64_t> Mask;
enum Shape { NIL = 0, CIRCLE = 1, BOX = 2 };

// The itemset record of Section 4.1: {mask, k, stop, supp, shape}.
struct Itemset {
  Mask mask;
  uint32_t k;
  uint32_t stop;
  uint64_t supp;
  Shape shape;
};

// One trace row per stop (loop iteration of Algorithm 2).
enum { TR_STEP, TR_STOP, TR_FIRST, TR_LAST, TR_DASHED, TR_PROMOTED, TR_PRUNED, TR_GENERATED,
       TR_SOLIDIFIED, TR_COLS };

struct Result {
  std::vector<std::vector<uint32_t>> sets;  // canonical order
  std::vector<uint64_t> supp;
  std::vector<uint64_t> trace;              // TR_COLS per row
  uint64_t tests = 0;                       // candidate-transaction tests
  uint64_t violations = 0;
};

uint32_t words_for(uint32_t m) { return (m + 63) / 64; }

// BitMask(T): bit p set iff item p in T (Section 4.1).
Mask bitmask(const uint32_t *it, uint64_t len, uint32_t W) {
  Mask w(W, 0);
  for (uint64_t j = 0; j < len; ++j) w[it[j] / 64] |= (uint64_t)1 << (it[j] % 64);
  return w;
}

// I subset-of T  <=>  BitMask(I) AND BitMask(T) = BitMask(I)   (Section 4.1)
bool contains(const Mask &T, const Mask &I) {
  for (size_t w = 0; w < I.size(); ++w)
    if ((I[w] & T[w]) != I[w]) return false;
  return true;
}

std::vector<uint32_t> items_of(const Mask &mk) {
  std::vector<uint32_t> v;
  for (size_t w = 0; w < mk.size(); ++w)
    for (int b = 0; b < 64; ++b)
      if ((mk[w] >> b) & 1) v.push_back((uint32_t)(w * 64 + b));
  return v;
}

bool canonical_less(const std::vector<uint32_t> &a, const std::vector<uint32_t> &b) {
  if (a.size() != b.size()) return a.size() < b.size();
  return a < b;
}

void finish(Result *r, std::vector<std::pair<std::vector<uint32_t>, uint64_t>> &L) {
  std::sort(L.begin(), L.end(), [](const std::pair<std::vector<uint32_t>, uint64_t> &x,
                                   const std::pair<std::vector<uint32_t>, uint64_t> &y) {
    return canonical_less(x.first, y.first);
  });
  for (auto &p : L) { r->sets.push_back(p.first); r->supp.push_back(p.second); }
}

std::vector<Mask> pack_all(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t W) {
  std::vector<Mask> B(n);
  for (uint64_t t = 0; t < n; ++t) B[t] = bitmask(items + row_ptr[t], row_ptr[t + 1] - row_ptr[t], W);
  return B;
}

// The DIC loop of Algorithm 2 after initialisation, shared by the ParallelDIC
// form (first pass done, DASHED holds the 2-itemset circles) and the classic
// form of Algorithm 1 (DASHED holds all 1-itemset circles).
void dic_loop(const std::vector<Mask> &B, uint64_t n, uint32_t m, uint32_t minsup, uint64_t M,
              std::vector<Itemset> &SOLID, std::vector<Itemset> &DASHED,
              std::map<Mask, uint64_t> &boxes, std::set<Mask> &ever, Result *r,
              uint64_t max_stops, bool superset_loop) {
  const uint32_t W = words_for(m);
  const uint64_t stop_max = (n + M - 1) / M;
  uint64_t stop = 0, step = 0;
  while (!DASHED.empty()) {
    if (max_stops && step == max_stops) break;  // timing samples only
    // Scan the database and rewind if necessary.
    ++step;
    stop = stop + 1;
    if (stop > stop_max) stop = 1;
    const uint64_t first = (stop - 1) * M;
    const uint64_t last = std::min(stop * M, n);  // exclusive
    uint64_t row[TR_COLS] = {0};
    row[TR_STEP] = step; row[TR_STOP] = stop; row[TR_FIRST] = first; row[TR_LAST] = last;
    row[TR_DASHED] = DASHED.size();

    // COUNTSUPPORT (Algorithm 3): every dashed itemset over the block.
    for (Itemset &I : DASHED) {
      I.stop = I.stop + 1;
      for (uint64_t t = first; t < last; ++t)
        if (contains(B[t], I.mask)) I.supp = I.supp + 1;
    }
    r->tests += (uint64_t)DASHED.size() * (last - first);

    // PRUNE (Algorithm 4) over the dashed circles.
    std::vector<size_t> promoted;
    for (size_t a = 0; a < DASHED.size(); ++a) {
      Itemset &I = DASHED[a];
      if (I.shape != CIRCLE) continue;
      if (I.supp >= minsup) {
        I.shape = BOX;  // move to Dashed Box
        boxes[I.mask] = step;
        promoted.push_back(a);
      } else {
        const uint64_t supp_max = I.supp + M * (stop_max - I.stop);
        if (supp_max < minsup) {
          I.shape = NIL;
          ++row[TR_PRUNED];
          for (size_t b = 0; superset_loop && b < DASHED.size(); ++b) {
            Itemset &J = DASHED[b];
            if (J.shape != CIRCLE) continue;
            if (contains(J.mask, I.mask)) {  // I.mask AND J.mask = I.mask
              J.shape = NIL;
              ++r->violations;  // only I itself could match, and it is NIL now
              ++row[TR_PRUNED];
            }
          }
        }
      }
    }
    row[TR_PROMOTED] = promoted.size();
    {
      std::vector<Itemset> keep;
      keep.reserve(DASHED.size());
      for (Itemset &I : DASHED)
        if (I.shape != NIL) keep.push_back(I);
      DASHED.swap(keep);
      // indices in `promoted` refer to the old vector; rebuild them as masks
    }

    // MAKECANDIDATES: immediate supersets C = I u {i} of the itemsets just
    // moved to Dashed Box whose every (|C|-1)-subset is a box.
    std::vector<Mask> newly;
    for (Itemset &I : DASHED)
      if (I.shape == BOX && boxes[I.mask] == step) newly.push_back(I.mask);
    std::set<Mask> fresh;
    std::vector<Mask> fresh_order;
    for (const Mask &A : newly) {
      for (uint32_t i = 0; i < m; ++i) {
        if ((A[i / 64] >> (i % 64)) & 1) continue;
        Mask C = A;
        C[i / 64] |= (uint64_t)1 << (i % 64);
        bool all_boxes = true;
        for (uint32_t j : items_of(C)) {
          Mask S = C;
          S[j / 64] &= ~((uint64_t)1 << (j % 64));
          if (boxes.find(S) == boxes.end()) { all_boxes = false; break; }
        }
        if (!all_boxes) continue;
        if (fresh.count(C)) continue;
        fresh.insert(C);
        fresh_order.push_back(C);
      }
    }
    for (const Mask &C : fresh_order) {
      if (ever.count(C)) ++r->violations;  // generated before
      ever.insert(C);
      Itemset J;
      J.mask = C;
      J.k = (uint32_t)items_of(C).size();
      J.stop = 0; J.supp = 0; J.shape = CIRCLE;
      DASHED.push_back(J);
    }
    row[TR_GENERATED] = fresh_order.size();

    // CHECKFULLPASS (Algorithm 5) over all of DASHED.
    {
      std::vector<Itemset> keep;
      keep.reserve(DASHED.size());
      for (Itemset &I : DASHED) {
        if (I.stop == stop_max) {
          if (I.supp >= minsup) I.shape = BOX;
          SOLID.push_back(I);
          ++row[TR_SOLIDIFIED];
        } else {
          keep.push_back(I);
        }
      }
      DASHED.swap(keep);
    }
    for (int c = 0; c < TR_COLS; ++c) r->trace.push_back(row[c]);
    (void)W;
  }
}

void collect(const std::vector<Itemset> &SOLID, Result *r) {
  std::vector<std::pair<std::vector<uint32_t>, uint64_t>> L;
  for (const Itemset &I : SOLID)
    if (I.shape == BOX) L.push_back({items_of(I.mask), I.supp});
  finish(r, L);
}

}  // namespace

extern "C" {

typedef struct Result oracle_result;

// BitMask of every row into words[n*W] (row-major), W = ceil(m/64).
int oracle_pack(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                uint64_t *words) {
  const uint32_t W = words_for(m);
  for (uint64_t t = 0; t < n; ++t) {
    Mask w = bitmask(items + row_ptr[t], row_ptr[t + 1] - row_ptr[t], W);
    std::memcpy(words + t * W, w.data(), W * sizeof(uint64_t));
  }
  return 0;
}

// ParallelDIC (Algorithm 2), serial.
// max_stops > 0 ends the loop after that many stops (a bounded timing sample;
// the itemsets are then incomplete). 0 runs to completion. superset_loop = 0
// skips the superset loop of Algorithm 4 (quadratic in |DASHED|; it never
// changes anything, which the pinned runs check by running it).
int oracle_dic(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
               uint32_t minsup, uint64_t M, uint64_t max_stops, int superset_loop,
               oracle_result **out) {
  *out = nullptr;
  if (m == 0 || minsup == 0 || M == 0) return -1;
  Result *r = new Result();
  const uint32_t W = words_for(m);
  if (n == 0) { *out = r; return 0; }
  std::vector<Mask> B = pack_all(row_ptr, items, n, W);

  // Initialise: SOLID holds the m 1-itemsets (shape NIL, stop 0, supp 0).
  std::vector<Itemset> SOLID, DASHED;
  for (uint32_t i = 0; i < m; ++i) {
    Itemset I;
    I.mask.assign(W, 0);
    I.mask[i / 64] |= (uint64_t)1 << (i % 64);
    I.shape = NIL; I.stop = 0; I.supp = 0; I.k = 1;
    SOLID.push_back(I);
  }
  // FIRSTPASS: count every 1-itemset over all n rows (like Algorithm 3).
  for (Itemset &I : SOLID)
    for (uint64_t t = 0; t < n; ++t)
      if (contains(B[t], I.mask)) I.supp = I.supp + 1;
  r->tests += (uint64_t)m * n;
  std::map<Mask, uint64_t> boxes;
  std::vector<Mask> L1;
  for (Itemset &I : SOLID) {
    I.shape = I.supp >= minsup ? BOX : CIRCLE;
    if (I.shape == BOX) { boxes[I.mask] = 0; L1.push_back(I.mask); }
  }
  // Candidate 2-itemsets: bitwise OR of every pair of frequent 1-itemsets.
  std::set<Mask> ever;
  for (size_t a = 0; a < L1.size(); ++a)
    for (size_t b = a + 1; b < L1.size(); ++b) {
      Itemset J;
      J.mask.resize(W);
      for (uint32_t w = 0; w < W; ++w) J.mask[w] = L1[a][w] | L1[b][w];
      J.k = 2; J.stop = 0; J.supp = 0; J.shape = CIRCLE;
      ever.insert(J.mask);
      DASHED.push_back(J);
    }
  dic_loop(B, n, m, minsup, M, SOLID, DASHED, boxes, ever, r, max_stops, superset_loop != 0);
  collect(SOLID, r);
  *out = r;
  return 0;
}

// Serial DIC of Algorithm 1: Dashed Circle starts with all 1-itemsets.
int oracle_dic_classic(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                       uint32_t minsup, uint64_t M, uint64_t max_stops, int superset_loop,
                       oracle_result **out) {
  *out = nullptr;
  if (m == 0 || minsup == 0 || M == 0) return -1;
  Result *r = new Result();
  const uint32_t W = words_for(m);
  if (n == 0) { *out = r; return 0; }
  std::vector<Mask> B = pack_all(row_ptr, items, n, W);
  std::vector<Itemset> SOLID, DASHED;
  std::set<Mask> ever;
  for (uint32_t i = 0; i < m; ++i) {
    Itemset I;
    I.mask.assign(W, 0);
    I.mask[i / 64] |= (uint64_t)1 << (i % 64);
    I.shape = CIRCLE; I.stop = 0; I.supp = 0; I.k = 1;
    ever.insert(I.mask);
    DASHED.push_back(I);
  }
  std::map<Mask, uint64_t> boxes;
  dic_loop(B, n, m, minsup, M, SOLID, DASHED, boxes, ever, r, max_stops, superset_loop != 0);
  collect(SOLID, r);
  *out = r;
  return 0;
}

// Apriori (Section 3): L1 by counting; C_k = joins of L_{k-1} members that
// share their first k-2 items, minus those with a (k-1)-subset outside
// L_{k-1}; each candidate counted by sorted-list inclusion over all rows.
int oracle_apriori(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                   uint32_t minsup, oracle_result **out) {
  *out = nullptr;
  if (m == 0 || minsup == 0) return -1;
  Result *r = new Result();
  std::vector<std::pair<std::vector<uint32_t>, uint64_t>> L;
  std::vector<uint64_t> c1(m, 0);
  for (uint64_t t = 0; t < n; ++t)
    for (uint64_t j = row_ptr[t]; j < row_ptr[t + 1]; ++j) c1[items[j]]++;
  std::vector<std::vector<uint32_t>> prev;
  for (uint32_t i = 0; i < m; ++i)
    if (c1[i] >= minsup) { prev.push_back({i}); L.push_back({{i}, c1[i]}); }
  while (!prev.empty()) {
    std::set<std::vector<uint32_t>> prevset(prev.begin(), prev.end());
    std::vector<std::vector<uint32_t>> cand;
    for (size_t a = 0; a < prev.size(); ++a)
      for (size_t b = a + 1; b < prev.size(); ++b) {
        const std::vector<uint32_t> &X = prev[a], &Y = prev[b];
        if (!std::equal(X.begin(), X.end() - 1, Y.begin())) continue;
        std::vector<uint32_t> C = X;
        C.push_back(Y.back());
        std::sort(C.begin(), C.end());
        bool ok = true;
        for (size_t d = 0; d < C.size() && ok; ++d) {
          std::vector<uint32_t> S;
          for (size_t e = 0; e < C.size(); ++e)
            if (e != d) S.push_back(C[e]);
          ok = prevset.count(S) > 0;
        }
        if (ok) cand.push_back(C);
      }
    std::vector<uint64_t> cnt(cand.size(), 0);
    for (uint64_t t = 0; t < n; ++t) {
      const uint32_t *b = items + row_ptr[t], *e = items + row_ptr[t + 1];
      for (size_t c = 0; c < cand.size(); ++c)
        if (std::includes(b, e, cand[c].begin(), cand[c].end())) cnt[c]++;
    }
    r->tests += (uint64_t)cand.size() * n;
    prev.clear();
    for (size_t c = 0; c < cand.size(); ++c)
      if (cnt[c] >= minsup) { prev.push_back(cand[c]); L.push_back({cand[c], cnt[c]}); }
    std::sort(prev.begin(), prev.end());
    uint64_t row[TR_COLS] = {0};
    row[TR_STEP] = r->trace.size() / TR_COLS + 1;
    row[TR_DASHED] = cand.size();
    row[TR_PROMOTED] = prev.size();
    for (int c = 0; c < TR_COLS; ++c) r->trace.push_back(row[c]);
  }
  finish(r, L);
  *out = r;
  return 0;
}

// Brute force: every non-empty subset X of {0..m-1} with support >= minsup,
// each row adding 1 to every sub-mask of its item mask. m <= 24.
int oracle_bruteforce(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                      uint32_t minsup, oracle_result **out) {
  *out = nullptr;
  if (m == 0 || m > 24 || minsup == 0) return -1;
  std::vector<uint32_t> cnt((size_t)1 << m, 0);
  for (uint64_t t = 0; t < n; ++t) {
    uint32_t T = 0;
    for (uint64_t j = row_ptr[t]; j < row_ptr[t + 1]; ++j) T |= 1u << items[j];
    for (uint32_t S = T; S != 0; S = (S - 1) & T) cnt[S]++;
  }
  Result *r = new Result();
  std::vector<std::pair<std::vector<uint32_t>, uint64_t>> L;
  for (uint32_t S = 1; S < ((uint32_t)1 << m); ++S)
    if (cnt[S] >= minsup) {
      std::vector<uint32_t> v;
      for (uint32_t i = 0; i < m; ++i)
        if ((S >> i) & 1) v.push_back(i);
      L.push_back({v, cnt[S]});
    }
  finish(r, L);
  *out = r;
  return 0;
}

// support(X) = number of rows containing every item of X, computed as the
// size of the intersection of the items' sorted row-id lists. Queries are
// CSR (q_off[nq+1], q_items); an empty query has support n.
int oracle_support(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                   const uint64_t *q_off, const uint32_t *q_items, uint64_t nq, uint64_t *supp) {
  std::vector<std::vector<uint32_t>> tid(m);
  for (uint64_t t = 0; t < n; ++t)
    for (uint64_t j = row_ptr[t]; j < row_ptr[t + 1]; ++j) tid[items[j]].push_back((uint32_t)t);
  for (uint64_t q = 0; q < nq; ++q) {
    if (q_off[q] == q_off[q + 1]) { supp[q] = n; continue; }
    bool bad = false;
    for (uint64_t j = q_off[q]; j < q_off[q + 1]; ++j) bad |= q_items[j] >= m;
    if (bad) return -1;
    std::vector<uint32_t> cur = tid[q_items[q_off[q]]];
    for (uint64_t j = q_off[q] + 1; j < q_off[q + 1] && !cur.empty(); ++j) {
      const std::vector<uint32_t> &o = tid[q_items[j]];
      std::vector<uint32_t> nx;
      std::set_intersection(cur.begin(), cur.end(), o.begin(), o.end(), std::back_inserter(nx));
      cur.swap(nx);
    }
    supp[q] = cur.size();
  }
  return 0;
}

// out[a*m + b] = number of rows containing both a and b (a != b); the
// diagonal holds the single-item counts.
int oracle_pair_supports(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                         uint32_t *out) {
  std::memset(out, 0, (size_t)m * m * sizeof(uint32_t));
  for (uint64_t t = 0; t < n; ++t) {
    const uint32_t *b = items + row_ptr[t];
    const uint64_t len = row_ptr[t + 1] - row_ptr[t];
    for (uint64_t x = 0; x < len; ++x) {
      out[(size_t)b[x] * m + b[x]]++;
      for (uint64_t y = x + 1; y < len; ++y) {
        out[(size_t)b[x] * m + b[y]]++;
        out[(size_t)b[y] * m + b[x]]++;
      }
    }
  }
  return 0;
}

uint64_t oracle_result_count(const oracle_result *r) { return r->sets.size(); }
uint64_t oracle_result_nitems(const oracle_result *r) {
  uint64_t s = 0;
  for (auto &v : r->sets) s += v.size();
  return s;
}
// k[count], items[nitems] (concatenated, ascending per set), supp[count]
void oracle_result_copy(const oracle_result *r, uint32_t *k, uint32_t *items, uint64_t *supp) {
  uint64_t p = 0;
  for (size_t i = 0; i < r->sets.size(); ++i) {
    k[i] = (uint32_t)r->sets[i].size();
    supp[i] = r->supp[i];
    for (uint32_t x : r->sets[i]) items[p++] = x;
  }
}
uint64_t oracle_result_trace_len(const oracle_result *r) { return r->trace.size() / TR_COLS; }
uint32_t oracle_trace_cols(void) { return TR_COLS; }
void oracle_result_trace(const oracle_result *r, uint64_t *rows) {
  if (!r->trace.empty()) std::memcpy(rows, r->trace.data(), r->trace.size() * sizeof(uint64_t));
}
uint64_t oracle_result_tests(const oracle_result *r) { return r->tests; }
uint64_t oracle_result_violations(const oracle_result *r) { return r->violations; }
void oracle_result_free(oracle_result *r) { delete r; }

}  // extern "C"
