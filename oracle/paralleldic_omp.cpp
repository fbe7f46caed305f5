// ParallelDIC on the host cores with OpenMP -- a CPU BASELINE for the
// benchmark, part of the test infrastructure (like the oracle beside it): the
// CUDA library never loads it and shares no code with it.
//
// It restates the paper's own parallel design (Section 4.2) rather than a
// GPU one:
//   * transactions and itemsets are bit masks of W = ceil(m/64) 64-bit words
//     (Section 4.1); the containment test is (I.mask AND T) == I.mask over all
//     W words, a loop the compiler vectorises;
//   * FIRSTPASS counts the 1-itemsets over all transactions like Algorithm 3,
//     then the Apriori join of the frequent items (bitwise OR of every pair)
//     fills Dashed Circle;
//   * COUNTSUPPORT (Algorithm 3) runs the itemset loop outside the
//     transaction loop (Figure 2) with `omp parallel for` over DASHED when it
//     holds at least as many itemsets as threads; otherwise (Figure 3) nested
//     parallelism: one outer thread per itemset, each forking
//     ceil(threads / |DASHED|) inner threads that reduce the count over the
//     block's transactions;
//   * PRUNE (Algorithm 4) and CHECKFULLPASS (Algorithm 5) are `omp parallel
//     for` over DASHED; MAKECANDIDATES joins the boxes (serial, as the paper
//     leaves it).
// Readings shared with the oracle: minsup is a count and frequent means >=;
// block s is [(s-1)M, min(sM, n)); the prune bound is supp + M*(stop_max -
// stop) in 64-bit; the new candidates of a stop are the itemsets of >= 3
// items whose subsets with one item fewer are all boxes and at least one of
// them was promoted at this stop; phase order COUNT, PRUNE, MAKECANDIDATES,
// CHECKFULLPASS. Algorithm 4's superset loop is left out: every subset of a
// lattice member is a box, so it can only ever match the pruned itemset
// itself (the oracle runs it and records that it never does more).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include <omp.h>

namespace {

enum Shape : uint8_t { NIL = 0, CIRCLE = 1, BOX = 2 };

struct Itemset {
  uint32_t off;    // first word of its mask in the mask pool
  uint32_t k;
  uint32_t stop;   // blocks counted so far
  uint64_t supp;
  Shape shape;
  uint32_t promo;  // stop number (global) at which it became a box
};

enum { TR_STEP, TR_STOP, TR_FIRST, TR_LAST, TR_DASHED, TR_PROMOTED, TR_PRUNED, TR_GENERATED,
       TR_SOLIDIFIED, TR_COLS };

}  // namespace

struct pdic_result {
  std::vector<std::vector<uint32_t>> sets;
  std::vector<uint64_t> supp;
  std::vector<uint64_t> trace;
  uint64_t tests = 0;
  int threads = 0;
};

// (I.mask AND T) == I.mask over W words.
static inline bool contains(const uint64_t *T, const uint64_t *I, uint32_t W) {
  uint64_t miss = 0;
  for (uint32_t w = 0; w < W; ++w) miss |= I[w] & ~T[w];
  return miss == 0;
}

// Sums `len` counters across the ranks of a sharded mine, in place (every
// rank calls it with its own partial counts and receives the totals);
// returns 0 on success.
typedef int (*pdic_reduce_fn)(void *ctx, uint64_t *counts, uint64_t len);

// The rows of block [first, last) that rank `rank` of `world` counts: an
// equal contiguous share of the block.
static inline void shard_of(uint64_t first, uint64_t last, int rank, int world, uint64_t *lo,
                            uint64_t *hi) {
  const uint64_t len = last - first;
  *lo = first + len * (uint64_t)rank / (uint64_t)world;
  *hi = first + len * (uint64_t)(rank + 1) / (uint64_t)world;
}

static int mine_impl(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                     uint32_t minsup, uint64_t M, uint64_t max_stops, int threads, int rank,
                     int world, pdic_reduce_fn reduce, void *ctx, pdic_result **out);

extern "C" {

// Mines rows given as CSR item lists with `threads` OpenMP threads (0 = the
// runtime's default). max_stops > 0 ends after that many stops (a bounded
// sample of the loop; the result is then incomplete). Returns 0, or -1 on an
// invalid argument.
int pdic_mine(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
              uint32_t minsup, uint64_t M, uint64_t max_stops, int threads, pdic_result **out) {
  return mine_impl(row_ptr, items, n, m, minsup, M, max_stops, threads, 0, 1, nullptr, nullptr,
                   out);
}

// Transaction-sharded mine, the data-distributed scheme of the paper's
// related work (Section 2: every processor counts the candidates over its
// own part of the transactions and the counts are summed): rank `rank` of
// `world` counts the first pass and every stop's dashed itemsets over its
// share of each block only, `reduce` sums those counters across the ranks
// (once for the first pass, once per stop), and every rank then runs PRUNE,
// MAKECANDIDATES and CHECKFULLPASS on the same totals, so all ranks hold
// the same lattice and return the single-rank result and trace. Returns 0,
// -1 on an invalid argument, -2 if `reduce` failed.
int pdic_mine_sharded(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                      uint32_t minsup, uint64_t M, uint64_t max_stops, int threads, int rank,
                      int world, pdic_reduce_fn reduce, void *ctx, pdic_result **out) {
  if (world < 1 || rank < 0 || rank >= world || (world > 1 && !reduce)) return -1;
  return mine_impl(row_ptr, items, n, m, minsup, M, max_stops, threads, rank, world, reduce, ctx,
                   out);
}

}  // extern "C"

static int mine_impl(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                     uint32_t minsup, uint64_t M, uint64_t max_stops, int threads, int rank,
                     int world, pdic_reduce_fn reduce, void *ctx, pdic_result **out) {
  if (!out || m == 0 || minsup == 0 || M == 0) return -1;
  *out = nullptr;
  const uint32_t W = (m + 63) / 64;
  if (threads <= 0) threads = omp_get_max_threads();
  omp_set_max_active_levels(2);
  pdic_result *r = new pdic_result();
  r->threads = threads;
  if (n == 0) { *out = r; return 0; }
  if (M > n) M = n;
  const uint64_t stop_max = (n + M - 1) / M;
  // BitMask of every transaction this rank counts (its share of each block)
  std::vector<uint64_t> B((size_t)n * W, 0);
  std::vector<uint8_t> mine((size_t)n, world == 1 ? 1 : 0);
  if (world > 1)
    for (uint64_t b = 0; b < stop_max; ++b) {
      uint64_t lo, hi;
      shard_of(b * M, std::min<uint64_t>((b + 1) * M, n), rank, world, &lo, &hi);
      for (uint64_t t = lo; t < hi; ++t) mine[t] = 1;
    }
#pragma omp parallel for num_threads(threads) schedule(static)
  for (int64_t t = 0; t < (int64_t)n; ++t)
    if (mine[t])
      for (uint64_t j = row_ptr[t]; j < row_ptr[t + 1]; ++j)
        B[(size_t)t * W + items[j] / 64] |= 1ull << (items[j] % 64);
  auto reduce_counts = [&](std::vector<uint64_t> &v) {
    if (world == 1 || v.empty()) return true;
    return reduce(ctx, v.data(), v.size()) == 0;
  };

  // FIRSTPASS: every 1-itemset over all transactions (Algorithm 3's form:
  // threads over itemsets, each scanning the transactions)
  std::vector<uint64_t> supp1(m, 0);
#pragma omp parallel for num_threads(threads) schedule(dynamic, 1)
  for (int64_t i = 0; i < (int64_t)m; ++i) {
    const uint32_t w = (uint32_t)i / 64;
    const uint64_t bit = 1ull << (i % 64);
    uint64_t c = 0;
    for (uint64_t t = 0; t < n; ++t) c += (B[(size_t)t * W + w] & bit) != 0;
    supp1[i] = c;
  }
  if (!reduce_counts(supp1)) { delete r; return -2; }
  r->tests = (uint64_t)m * n;
  std::vector<uint32_t> L1;
  for (uint32_t i = 0; i < m; ++i)
    if (supp1[i] >= minsup) {
      L1.push_back(i);
      r->sets.push_back({i});
      r->supp.push_back(supp1[i]);
    }

  std::vector<uint64_t> pool;  // masks of every itemset ever created
  std::vector<Itemset> DASHED, SOLID;
  auto new_mask = [&]() {
    const uint32_t off = (uint32_t)pool.size();
    pool.resize(pool.size() + W, 0);
    return off;
  };
  // pair join: bitwise OR of every pair of frequent 1-itemsets
  for (size_t a = 0; a < L1.size(); ++a)
    for (size_t b = a + 1; b < L1.size(); ++b) {
      const uint32_t off = new_mask();
      pool[off + L1[a] / 64] |= 1ull << (L1[a] % 64);
      pool[off + L1[b] / 64] |= 1ull << (L1[b] % 64);
      DASHED.push_back({off, 2, 0, 0, CIRCLE, 0});
    }
  // every box ever promoted (itemsets of >= 2 items), by mask bytes: its
  // promotion stop (boxes never change shape, solid or not)
  std::unordered_map<std::string, uint32_t> boxes;
  auto key_of = [&](const uint64_t *mk) {
    return std::string(reinterpret_cast<const char *>(mk), (size_t)W * 8);
  };

  uint64_t stop = 0, step = 0;
  std::vector<uint64_t> cand(W), sub(W);
  while (!DASHED.empty()) {
    if (max_stops && step == max_stops) break;
    ++step;
    stop = stop + 1;
    if (stop > stop_max) stop = 1;
    const uint64_t first = (stop - 1) * M, last = std::min<uint64_t>(stop * M, n);
    uint64_t row[TR_COLS] = {0};
    row[TR_STEP] = step; row[TR_STOP] = stop; row[TR_FIRST] = first; row[TR_LAST] = last;
    row[TR_DASHED] = DASHED.size();
    r->tests += (uint64_t)DASHED.size() * (last - first);

    // COUNTSUPPORT (Algorithm 3, Figures 2 and 3) over this rank's share of
    // the block, then (sharded) one sum of the counters across the ranks
    uint64_t lo = first, hi = last;
    if (world > 1) shard_of(first, last, rank, world, &lo, &hi);
    const int64_t D = (int64_t)DASHED.size();
    std::vector<uint64_t> part((size_t)D, 0);
    if (D >= threads) {
#pragma omp parallel for num_threads(threads) schedule(dynamic, 64)
      for (int64_t q = 0; q < D; ++q) {
        const uint64_t *mk = &pool[DASHED[q].off];
        uint64_t c = 0;
        for (uint64_t t = lo; t < hi; ++t) c += contains(&B[(size_t)t * W], mk, W);
        part[q] = c;
      }
    } else {
      const int inner = (threads + (int)D - 1) / (int)D;
#pragma omp parallel for num_threads((int)D) schedule(static, 1)
      for (int64_t q = 0; q < D; ++q) {
        const uint64_t *mk = &pool[DASHED[q].off];
        uint64_t c = 0;
#pragma omp parallel for num_threads(inner) reduction(+ : c) schedule(static)
        for (int64_t t = (int64_t)lo; t < (int64_t)hi; ++t)
          c += contains(&B[(size_t)t * W], mk, W);
        part[q] = c;
      }
    }
    if (!reduce_counts(part)) { delete r; return -2; }
    for (int64_t q = 0; q < D; ++q) {
      DASHED[q].stop += 1;
      DASHED[q].supp += part[q];
    }

    // PRUNE (Algorithm 4)
    uint64_t promoted = 0, pruned = 0;
#pragma omp parallel for num_threads(threads) schedule(static) reduction(+ : promoted, pruned)
    for (int64_t q = 0; q < D; ++q) {
      Itemset &I = DASHED[q];
      if (I.shape != CIRCLE) continue;
      if (I.supp >= minsup) {
        I.shape = BOX;
        I.promo = (uint32_t)step;
        ++promoted;
      } else if (I.supp + M * (stop_max - I.stop) < minsup) {
        I.shape = NIL;
        ++pruned;
      }
    }
    std::vector<Itemset> newly;
    for (const Itemset &I : DASHED)
      if (I.shape == BOX && I.promo == step) {
        newly.push_back(I);
        boxes.emplace(key_of(&pool[I.off]), (uint32_t)step);
      }
    {
      std::vector<Itemset> keep;
      keep.reserve(DASHED.size());
      for (const Itemset &I : DASHED)
        if (I.shape != NIL) keep.push_back(I);
      DASHED.swap(keep);
    }

    // MAKECANDIDATES: C = A OR {i} for A promoted at this stop and a
    // frequent item i outside A, kept when every subset of C with one item
    // fewer is a box; of C's parents promoted at this stop only the one
    // missing the smallest item emits it
    uint64_t generated = 0;
    for (const Itemset &A : newly) {
      const uint64_t *a = &pool[A.off];
      for (uint32_t i : L1) {
        if ((a[i / 64] >> (i % 64)) & 1) continue;
        std::memcpy(cand.data(), a, (size_t)W * 8);
        cand[i / 64] |= 1ull << (i % 64);
        bool ok = true;
        for (uint32_t w = 0; w < W && ok; ++w)
          for (uint64_t x = cand[w]; x && ok; x &= x - 1) {
            const uint32_t j = w * 64 + (uint32_t)__builtin_ctzll(x);
            if (j == i) continue;
            sub = cand;
            sub[j / 64] &= ~(1ull << (j % 64));
            auto it = boxes.find(key_of(sub.data()));
            if (it == boxes.end() || (j < i && it->second == step)) ok = false;
          }
        if (!ok) continue;
        const uint32_t off = new_mask();
        std::memcpy(&pool[off], cand.data(), (size_t)W * 8);
        DASHED.push_back({off, A.k + 1, 0, 0, CIRCLE, 0});
        ++generated;
      }
    }

    // CHECKFULLPASS (Algorithm 5)
    const int64_t D2 = (int64_t)DASHED.size();
    std::vector<uint8_t> full(D2, 0);
#pragma omp parallel for num_threads(threads) schedule(static)
    for (int64_t q = 0; q < D2; ++q) {
      Itemset &I = DASHED[q];
      if (I.stop == stop_max) {
        if (I.supp >= minsup) I.shape = BOX;
        full[q] = 1;
      }
    }
    uint64_t solidified = 0;
    {
      std::vector<Itemset> keep;
      keep.reserve(DASHED.size());
      for (int64_t q = 0; q < D2; ++q) {
        if (full[q]) { SOLID.push_back(DASHED[q]); ++solidified; }
        else keep.push_back(DASHED[q]);
      }
      DASHED.swap(keep);
    }
    row[TR_PROMOTED] = promoted;
    row[TR_PRUNED] = pruned;
    row[TR_GENERATED] = generated;
    row[TR_SOLIDIFIED] = solidified;
    r->trace.insert(r->trace.end(), row, row + TR_COLS);
  }
  // L: the frequent 1-itemsets and the solid boxes, size then lexicographic
  for (const Itemset &I : SOLID) {
    if (I.shape != BOX) continue;
    std::vector<uint32_t> v;
    for (uint32_t w = 0; w < W; ++w)
      for (uint64_t x = pool[I.off + w]; x; x &= x - 1)
        v.push_back(w * 64 + (uint32_t)__builtin_ctzll(x));
    r->sets.push_back(std::move(v));
    r->supp.push_back(I.supp);
  }
  std::vector<size_t> order(r->sets.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](size_t x, size_t y) {
    const auto &a = r->sets[x], &b = r->sets[y];
    return a.size() != b.size() ? a.size() < b.size() : a < b;
  });
  std::vector<std::vector<uint32_t>> sets;
  std::vector<uint64_t> sp;
  for (size_t i : order) { sets.push_back(r->sets[i]); sp.push_back(r->supp[i]); }
  r->sets.swap(sets);
  r->supp.swap(sp);
  *out = r;
  return 0;
}

extern "C" {

uint64_t pdic_result_count(const pdic_result *r) { return r->sets.size(); }
uint64_t pdic_result_nitems(const pdic_result *r) {
  uint64_t t = 0;
  for (const auto &v : r->sets) t += v.size();
  return t;
}
void pdic_result_copy(const pdic_result *r, uint32_t *k, uint32_t *items, uint64_t *supp) {
  uint64_t p = 0;
  for (size_t i = 0; i < r->sets.size(); ++i) {
    k[i] = (uint32_t)r->sets[i].size();
    for (uint32_t x : r->sets[i]) items[p++] = x;
    supp[i] = r->supp[i];
  }
}
uint64_t pdic_result_trace_len(const pdic_result *r) { return r->trace.size() / TR_COLS; }
void pdic_result_trace(const pdic_result *r, uint64_t *rows) {
  if (!r->trace.empty()) std::memcpy(rows, r->trace.data(), r->trace.size() * 8);
}
uint64_t pdic_result_tests(const pdic_result *r) { return r->tests; }
int pdic_result_threads(const pdic_result *r) { return r->threads; }
void pdic_result_free(pdic_result *r) { delete r; }

}  // extern "C"
