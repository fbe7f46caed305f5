// Device-side helpers of the lattice shared by the count and lattice kernels:
// the box set (open addressing over candidate indices) and the PRUNE /
// promotion rule of Algorithm 4 applied to one record.
#pragma once
#include <cstdint>

#include "dic_internal.cuh"

namespace dic {

// Hash of a mask = final mix of the sum over words of hterm(word, index).
// The sum form lets MAKECANDIDATES derive the hash of C \ {j} from that of
// the parent in O(1).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t hterm(uint64_t w, uint32_t i) {
  return mix64(w + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1));
}
__device__ __forceinline__ uint32_t hslot_of(uint64_t sum, uint32_t hcap) {
  return (uint32_t)(mix64(sum ^ 0x5851F42D4C957F2Dull) & (uint64_t)(hcap - 1));
}
__device__ __forceinline__ uint64_t mask_hash_sum(const uint64_t *key, uint32_t wc) {
  uint64_t sum = 0;
  for (uint32_t i = 0; i < wc; ++i) sum += hterm(key[i], i);
  return sum;
}

// Insert record c (a box) into the box set. Records are inserted once, so a
// thread that finds a slot taken probes on; callers guarantee a load factor
// <= 1/2, so a free slot exists.
__device__ __forceinline__ void box_insert(const Lattice &L, uint32_t c, uint64_t sum) {
  uint32_t slot = hslot_of(sum, L.hcap);
  for (uint32_t probe = 0; probe < L.hcap; ++probe) {
    if (atomicCAS(&L.hslot[slot], 0u, c + 1) == 0u) return;
    slot = (slot + 1) & (L.hcap - 1);
  }
}

// The box whose mask is A | br (in word wr) with bit bj of word wj cleared,
// or 0 if absent; otherwise its promotion stop + 1.
__device__ __forceinline__ uint32_t box_lookup(const Lattice &L, const uint64_t *A, uint32_t wr,
                                               uint64_t br, uint32_t wj, uint64_t bj,
                                               uint64_t sum) {
  uint32_t slot = hslot_of(sum, L.hcap);
  for (uint32_t probe = 0; probe < L.hcap; ++probe) {
    const uint32_t v = L.hslot[slot];
    if (v == 0) return 0;
    const uint64_t *key = L.cmask + (uint64_t)(v - 1) * L.wc;
    bool eq = true;
    for (uint32_t i = 0; i < L.wc && eq; ++i) {
      uint64_t s = A[i];
      if (i == wr) s |= br;
      if (i == wj) s &= ~bj;
      eq = key[i] == s;
    }
    if (eq) return L.cpromo[v - 1] + 1;
    slot = (slot + 1) & (L.hcap - 1);
  }
  return 0;
}

// Record a promotion of record c at stop g: shape, promotion stop, the list
// MAKECANDIDATES reads, and (when `insert`) the box set.
__device__ __forceinline__ void promote_record(const Lattice &L, Ctrl *C, uint32_t c, uint32_t g,
                                               bool insert) {
  // the size and first two ranks MAKECANDIDATES needs, loaded beside the
  // slot reservation
  const uint32_t k = L.ck[c];
  const uint32_t r01 = *reinterpret_cast<const uint32_t *>(L.cranks + (uint64_t)c * KRMAX);
  L.cshape[c] = SH_BOX;
  L.cpromo[c] = g;
  const uint32_t at = atomicAdd(&C->n_newbox, 1u);
  L.newbox[at] = c;
  L.newinfo[at] = (uint64_t)k | ((uint64_t)(r01 & 0xFFFFu) << 8) | ((uint64_t)(r01 >> 16) << 24);
  if (insert) {
    const uint64_t sum = mask_hash_sum(L.cmask + (uint64_t)c * L.wc, L.wc);
    L.newhash[at] = sum;
    box_insert(L, c, sum);
  }
}

// Algorithm 4 for one dashed record after its count at stop g, given its
// new support s: a circle with s >= minsup becomes a box; a circle whose
// bound s + M * (stop_max - stop) is below minsup is erased (stop = g -
// birth, the blocks counted so far). Tallies records completing their full
// pass (every live one is a box there). Returns nothing; updates tallies.
// This form takes the record's shape and birth stop already loaded.
__device__ __forceinline__ void settle_loaded(const Lattice &L, Ctrl *C, uint32_t c, uint8_t sh,
                                              uint32_t birth, uint32_t s, uint32_t g,
                                              bool insert, uint32_t &pruned, uint32_t &solid) {
  if (sh == SH_NIL) return;
  const uint32_t age = g - birth;
  if (sh == SH_CIRCLE) {
    if (s >= L.minsup) {
      promote_record(L, C, c, g, insert);
    } else if ((uint64_t)s + L.M * (uint64_t)(L.stop_max - age) < (uint64_t)L.minsup) {
      L.cshape[c] = SH_NIL;
      ++pruned;
      return;
    }
  }
  if (age == L.stop_max) ++solid;
}

__device__ __forceinline__ void settle_record(const Lattice &L, Ctrl *C, uint32_t c, uint32_t s,
                                              uint32_t g, bool insert, uint32_t &pruned,
                                              uint32_t &solid) {
  const uint8_t sh = L.cshape[c];
  if (sh == SH_NIL) return;
  settle_loaded(L, C, c, sh, L.cbirth[c], s, g, insert, pruned, solid);
}

// apply_pair_events (below) with the stop's event range already read
// (ev[0..2] = first and end index into ev_list, pairs dropped at g); thread
// 0 also adds the pair boxes completing their pass at stop_max.
__device__ __forceinline__ void apply_pair_events_range(const Lattice &L, Ctrl *C, uint32_t g,
                                                        const uint32_t ev[3], uint64_t tid,
                                                        uint64_t nthreads, uint32_t &pruned,
                                                        uint32_t &solid) {
  if (!L.pair_events || g > L.stop_max) return;
  for (uint64_t i = ev[0] + tid; i < ev[1]; i += nthreads)
    promote_record(L, C, L.ev_list[i], g, false);
  if (tid == 0) {
    pruned += ev[2];
    if (g == L.stop_max) solid += L.ev_pruned[0];
  }
}

// Stop g's precomputed PRUNE outcome for the pair cohort (Lattice
// pair_events): the pairs listed for g are promoted (box set insert, the
// list MAKECANDIDATES reads); the pairs dropped by the bound at g, and at
// stop_max the pair boxes completing their pass, are added to the caller's
// tallies by thread 0. Threads tid = 0 .. nthreads-1 share the work.
// The pairs are not inserted into the box set: with the first pass's
// lexicographic pair records (the only case with pair events),
// MAKECANDIDATES reads a pair's shape and promotion stop from its record and
// probes the box set only for subsets of three or more items.
__device__ __forceinline__ void apply_pair_events(const Lattice &L, Ctrl *C, uint32_t g,
                                                  uint64_t tid, uint64_t nthreads,
                                                  uint32_t &pruned, uint32_t &solid) {
  if (!L.pair_events || g > L.stop_max) return;
  const uint32_t ev[3] = {L.ev_off[g], L.ev_off[g + 1], L.ev_pruned[g]};
  apply_pair_events_range(L, C, g, ev, tid, nthreads, pruned, solid);
}

// MAKECANDIDATES for one (record promoted at g, rank r) pair: C = A | r is
// emitted iff every C \ {j} is a box and no j < r has C \ {j} promoted at g
// (the canonical parent). New records go to base + n_gen; past the capacity
// the stop stalls (ST_CAND) and nothing is written.
//
// First a necessary condition read straight from the pair cohort: C \ {j}
// for j in A other than a (a = A's first or second rank) contains {a, r},
// and every subset of a box is a box, so the pair records {a0, r} and
// {a1, r} must both be boxes. Most ranks r fail it with two loads and no
// probe of the box set; for a pair A those two records are all of C's
// other subsets, and the box set is not probed at all. (Only where the pair
// records are the first pass's complete lexicographic join.)
__device__ __forceinline__ void gen_candidate(const Lattice &L, Ctrl *C, uint32_t p, uint32_t r,
                                              uint32_t g, uint32_t base) {
  const uint32_t wc = L.wc;
  const uint32_t cA = L.newbox[p];
  const uint64_t info = L.newinfo[p];
  const uint32_t kA = (uint32_t)(info & 0xFFu);
  if (L.pairs_lex && kA >= 2) {
    const uint32_t a0 = (uint32_t)(info >> 8) & 0xFFFFu, a1 = (uint32_t)(info >> 24) & 0xFFFFu;
    if (r == a0 || r == a1) return;  // r in A
    const uint64_t l1 = L.l1;
    const uint64_t i0 = r < a0 ? pair_record(r, a0, l1) : pair_record(a0, r, l1);
    const uint64_t i1 = r < a1 ? pair_record(r, a1, l1) : pair_record(a1, r, l1);
    // promotion stops (~0: not a box; a stop after g: not a box yet)
    const uint32_t p0 = L.cpromo[i0], p1 = L.cpromo[i1];
    if (p0 > g || p1 > g) return;
    if (kA == 2) {
      // A = {a0, a1}: the 2-subsets of C other than A are the pair records
      // {a1, r} = C \ {a0} and {a0, r} = C \ {a1}, both boxes by the check
      // above, so only the canonical-parent rule remains (no box-set probe)
      if (a0 < r && p1 == g) return;
      if (a1 < r && p0 == g) return;
      const uint32_t pos = base + (uint32_t)atomicAdd(&C->gen_ticket, 1ull);
      if (pos >= L.cap) {
        C->stall = ST_CAND;
        return;
      }
      const uint32_t lo = r < a0 ? r : a0, hi = r > a1 ? r : a1;
      const uint32_t mid = r < a0 ? a0 : (r > a1 ? a1 : r);
      for (uint32_t i = 0; i < wc; ++i) {
        uint64_t x = 0;
        if ((lo >> 6) == i) x |= 1ull << (lo & 63);
        if ((mid >> 6) == i) x |= 1ull << (mid & 63);
        if ((hi >> 6) == i) x |= 1ull << (hi & 63);
        L.cmask[(uint64_t)pos * wc + i] = x;
      }
      uint16_t *rk = L.cranks + (uint64_t)pos * KRMAX;
      rk[0] = (uint16_t)lo; rk[1] = (uint16_t)mid; rk[2] = (uint16_t)hi;
      L.csupp[pos] = 0;
      L.cbirth[pos] = g;
      L.cshape[pos] = SH_CIRCLE;
      L.cpromo[pos] = ~0u;
      L.ck[pos] = 3;
      atomicMax(&C->max_k, 3u);
      return;
    }
  }  // (classic DIC, or a 1-itemset parent: the box-set probes below decide)
  const uint64_t *A = L.cmask + (uint64_t)cA * wc;
  const uint32_t wr = r >> 6;
  const uint64_t br = 1ull << (r & 63);
  const uint64_t Awr = A[wr];
  if (Awr & br) return;
  const uint64_t sumC = L.newhash[p] - hterm(Awr, wr) + hterm(Awr | br, wr);
  uint32_t k = 0;
  for (uint32_t i = 0; i < wc; ++i) {
    uint64_t x = A[i];
    const uint64_t Ci = i == wr ? (A[i] | br) : A[i];
    while (x) {
      const uint32_t b = (uint32_t)(__ffsll((long long)x) - 1);
      x &= x - 1;
      ++k;
      const uint64_t bj = 1ull << b;
      const uint64_t sumS = sumC - hterm(Ci, i) + hterm(Ci & ~bj, i);
      // (v = promotion stop + 1; the event-driven loop inserts boxes before
      // their promotion stop, which do not count until then)
      const uint32_t v = box_lookup(L, A, wr, br, i, bj, sumS);
      if (v == 0 || v > g + 1 || (i * 64 + b < r && v == g + 1)) return;
    }
  }
  const uint32_t pos = base + (uint32_t)atomicAdd(&C->gen_ticket, 1ull);
  if (pos >= L.cap) {
    C->stall = ST_CAND;
    return;
  }
  uint32_t q = 0;
  uint16_t *rk = L.cranks + (uint64_t)pos * KRMAX;
  for (uint32_t i = 0; i < wc; ++i) {
    const uint64_t x = i == wr ? (A[i] | br) : A[i];
    L.cmask[(uint64_t)pos * wc + i] = x;
    for (uint64_t y = x; y && q < KRMAX; y &= y - 1)
      rk[q++] = (uint16_t)(i * 64 + __ffsll((long long)y) - 1);
  }
  L.csupp[pos] = 0;
  L.cbirth[pos] = g;
  L.cshape[pos] = SH_CIRCLE;
  L.cpromo[pos] = ~0u;
  L.ck[pos] = (uint8_t)(k + 1 < 255 ? k + 1 : 255);
  atomicMax(&C->max_k, k + 1);
}

// End of stop g for one query: trace row, test count, the new cohort,
// CHECKFULLPASS (cohorts whose full pass is complete leave the window [head,
// tail)), |DASHED| and the loop test of Algorithm 2.
__device__ __forceinline__ void finish_stop_with(const Lattice &L, Ctrl *C, Ctrl &c);

__device__ __forceinline__ void finish_stop(const Lattice &L, Ctrl *C) {
  // one copy of the loop state in registers (independent loads, one round
  // trip)
  Ctrl c = *C;
  finish_stop_with(L, C, c);
}

// finish_stop from a copy of the loop state taken by the caller (with the
// stop's final candidate count); every field this stop changes is stored
// once at the end, and the caller's copy is brought to the same state.
__device__ __forceinline__ void finish_stop_with(const Lattice &L, Ctrl *C, Ctrl &c) {
  const uint32_t g = c.step;
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  if (c.n_trace >= L.tcap) {
    C->error = 4;  // DIC_ECAPACITY
    C->done = 1;
    c.error = 4;
    c.done = 1;
    return;
  }
  unsigned long long *row = L.trace + (uint64_t)c.n_trace * TRACE_COLS;
  row[0] = g; row[1] = stop; row[2] = first; row[3] = last;
  const uint32_t n_gen = n_gen_of(c);
  row[4] = c.n_live; row[5] = c.n_newbox; row[6] = c.n_pruned; row[7] = n_gen;
  row[8] = c.n_solid;
  if (L.trace_work) L.trace_work[c.n_trace] = c.work;
  uint32_t n_cohorts = c.n_cohorts;
  if (n_gen) {
    L.cohort_start[n_cohorts] = c.tail;
    L.cohort_birth[n_cohorts] = g;
    n_cohorts += 1;
    C->last_birth = g;
    c.last_birth = g;
  }
  const uint32_t tail = c.tail + n_gen;
  const uint32_t n_live = c.n_live - c.n_pruned - c.n_solid + n_gen;
  // CHECKFULLPASS: cohorts whose full pass ends with this stop leave the
  // window (a cohort born now never does: its birth + stop_max > g)
  // (head = the first remaining cohort's start; the new cohort, if any,
  // starts at the old tail, and so does an empty window)
  // (the oldest live cohort's birth is kept in the loop state, so a stop
  // that retires nothing reads no cohort record)
  uint32_t ch = c.cohort_head, head = c.head, hb = c.head_birth;
  if (hb + L.stop_max <= g) {
    head = c.tail;  // every old cohort retired: the window starts at the new one
    hb = g;
    while (ch < c.n_cohorts) {
      const uint32_t birth = L.cohort_birth[ch], start = L.cohort_start[ch];
      if (birth + L.stop_max > g) { head = start; hb = birth; break; }
      ++ch;
    }
  }
  if (c.n_newbox) c.last_promo = g;
  c.tests = c.tests + (unsigned long long)c.n_live * (last - first);
  c.n_cohorts = n_cohorts;
  c.tail = tail;
  c.hash_used = c.hash_used + c.n_newbox;
  c.n_live = n_live;
  c.cohort_head = ch;
  c.head = head;
  c.head_birth = hb;
  c.n_newbox = 0; c.n_pruned = 0; c.n_solid = 0; c.gen_ticket = 0;
  c.n_trace = c.n_trace + 1;
  c.step = g + 1;
  C->tests = c.tests;
  C->n_cohorts = c.n_cohorts;
  C->tail = c.tail;
  C->hash_used = c.hash_used;
  C->n_live = c.n_live;
  C->cohort_head = c.cohort_head;
  C->head = c.head;
  C->head_birth = c.head_birth;
  C->n_newbox = 0; C->n_pruned = 0; C->n_solid = 0; C->gen_ticket = 0;
  C->last_promo = c.last_promo;
  C->n_trace = c.n_trace;
  C->step = c.step;
  if (n_live == 0) {
    C->done = 1;
    c.done = 1;
  }
}


// Transpose a 32x32 bit block held one row per lane (bit b of lane t's word
// = element (t, b)) so that lane b ends with column b (bit t = element (t,
// b)). Five exchange stages: at distance j, the j x j off-diagonal
// sub-blocks of every 2j x 2j block swap places.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t lo_masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const uint32_t j = 16u >> st, mlo = lo_masks[st];
    const uint32_t v = __shfl_xor_sync(0xffffffffu, x, j);
    x = (lane & j) ? ((x & ~mlo) | ((v >> j) & mlo)) : ((x & mlo) | ((v << j) & ~mlo));
  }
  return x;
}

// BITSLICE column stride of a tile row (words): TW + 4 for TW = 8, 16 and TW
// for TW = 4, so rows start on 16-byte boundaries and eight threads reading
// consecutive ranks with 128-bit loads hit distinct banks.
__host__ __device__ constexpr uint32_t bs_stride(int tw) { return tw == 4 ? 4u : (uint32_t)tw + 4u; }

// Transpose the block of stop g into its column buffer: warp `wid`
// of `nwarps` handles (32-row word w, mask word j) items; bit j' of the
// result is row first+32w+j'. Out-of-range rows read as 0. An index outside
// V (an internal sizing error) is recorded in Ctrl.error and skipped.
__device__ __forceinline__ void slice_block_warps(const Lattice &L, uint32_t g, uint64_t wid,
                                                  uint64_t nwarps) {
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  const uint32_t tw = L.tw, l1p = L.l1p, st = bs_stride((int)tw);
  const uint32_t nw32 = (uint32_t)((last - first + 31) / 32);
  const uint32_t ntiles = (nw32 + tw - 1) / tw;
  const uint32_t wc = L.wc;
  const uint32_t lane = threadIdx.x & 31;
  uint32_t *V = vcols(L, g);
  const uint64_t items = (uint64_t)ntiles * tw * wc;
  for (uint64_t it = wid; it < items; it += nwarps) {
    const uint32_t w = (uint32_t)(it / wc), j = (uint32_t)(it % wc);
    const uint64_t row = first + 32ull * w + lane;
    const uint64_t x = (w < nw32 && row < last) ? __ldg(L.rows + row * wc + j) : 0ull;
    // lane b gets the 32 rows' bits of ranks 64j+b (lo) and 64j+32+b (hi)
    const uint32_t lo = warp_transpose32((uint32_t)x);
    const uint32_t hi = warp_transpose32((uint32_t)(x >> 32));
    const uint32_t t = w / tw, wi = w % tw;
    const uint32_t r0 = j * 64 + lane, r1 = r0 + 32;
    const uint64_t i0 = ((uint64_t)t * l1p + r0) * st + wi, i1 = ((uint64_t)t * l1p + r1) * st + wi;
    if ((r0 < l1p && i0 >= L.vwords) || (r1 < l1p && i1 >= L.vwords)) {
      L.ctrl->error = DIC_INTERNAL_BOUNDS;
      continue;
    }
    if (r0 < l1p) V[i0] = lo;
    if (r1 < l1p) V[i1] = hi;
  }
}

}  // namespace dic
