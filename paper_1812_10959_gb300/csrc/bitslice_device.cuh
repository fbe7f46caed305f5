// BITSLICE count body shared by the single-query and the batched kernels.
#pragma once
#include <cstdint>

#include "dic_internal.cuh"
#include "lattice_device.cuh"

namespace dic {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_1() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// Marker in the per-chunk size array for a record counted elsewhere.
constexpr uint8_t KSKIP = 255;

// Checks a count launch makes before changing anything for a query: every
// dashed itemset fits KRE ranks, and the box set has room for every live
// record to be promoted. Reads only values no count kernel changes, so all
// CTAs of a launch decide alike. `report` lets one thread raise the stall.
template <int KRE>
__device__ __forceinline__ bool bs_checks_v(const Lattice &L, Ctrl *C, uint32_t max_k,
                                            uint32_t hash_used, uint32_t n_live, bool report) {
  if (max_k > (uint32_t)KRE) {
    if (report && threadIdx.x == 0) C->stall = ST_WIDTH;
    return false;
  }
  if ((uint64_t)(hash_used + n_live) * 2 > L.hcap) {
    if (report && threadIdx.x == 0) C->stall = ST_HASH_COUNT;
    return false;
  }
  return true;
}
template <int KRE>
__device__ __forceinline__ bool bs_checks(const Lattice &L, Ctrl *C, bool report) {
  return bs_checks_v<KRE>(L, C, C->max_k, C->hash_used, C->n_live, report);
}

// The loop-state fields a stop kernel decides on, read in one round of
// independent loads (none of them changes while a count kernel runs).
struct StopState {
  uint32_t stall, done, step, head, tail, max_k, hash_used, n_live;
};
__device__ __forceinline__ StopState load_stop_state(const Ctrl *C) {
  StopState s;
  s.stall = C->stall; s.done = C->done; s.step = C->step; s.head = C->head;
  s.tail = C->tail; s.max_k = C->max_k; s.hash_used = C->hash_used; s.n_live = C->n_live;
  return s;
}

// The same, read by one thread per CTA and broadcast through shared memory
// together with the stop's pair-event range (lines every warp of a large
// grid would otherwise request from L2 at once, which serialises there).
// ev[0..2] = first and end index of the stop's promoted pairs and the
// number of pairs dropped at the stop (zeros without pair events). The
// whole CTA must call this.
__device__ __forceinline__ StopState cta_stop_state(const Lattice &L, const Ctrl *C,
                                                    uint32_t ev[3]) {
  __shared__ StopState s_st;
  __shared__ uint32_t s_ev[3];
  if (threadIdx.x == 0) {
    const StopState st = load_stop_state(C);
    // both slots, loaded with the rest (no load waits on the stop number)
    uint32_t es[2], en[6];
#pragma unroll
    for (int i = 0; i < 2; ++i) es[i] = C->ev_stop[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) en[i] = C->ev_next[i];
    uint32_t e0 = 0, e1 = 0, e2 = 0;
    if (L.pair_events && st.step <= L.stop_max && !st.stall && !st.done) {
      const uint32_t sl = st.step & 1u;
      if (es[sl] == st.step) {  // set by the previous stop's count
        e0 = en[3 * sl]; e1 = en[3 * sl + 1]; e2 = en[3 * sl + 2];
      } else {
        e0 = L.ev_off[st.step];
        e1 = L.ev_off[st.step + 1];
        e2 = L.ev_pruned[st.step];
      }
    }
    s_st = st;
    s_ev[0] = e0; s_ev[1] = e1; s_ev[2] = e2;
  }
  __syncthreads();
  ev[0] = s_ev[0]; ev[1] = s_ev[1]; ev[2] = s_ev[2];
  return s_st;
}

// One thread of the count kernel of stop g records the next stop's pair
// event range in the loop state (off the critical path of that stop).
__device__ __forceinline__ void stage_next_events(const Lattice &L, Ctrl *C, uint32_t g) {
  if (!L.pair_events || g + 1 > L.stop_max) return;
  const uint32_t e0 = L.ev_off[g + 1], e1 = L.ev_off[g + 2], e2 = L.ev_pruned[g + 1];
  const uint32_t sl = (g + 1) & 1u;
  C->ev_next[3 * sl] = e0; C->ev_next[3 * sl + 1] = e1; C->ev_next[3 * sl + 2] = e2;
  C->ev_stop[sl] = g + 1;
}

// 32-row words and tiles of stop g's block; false (error recorded) if they
// would not fit the column buffer.
template <int TW>
__device__ __forceinline__ bool bs_block_tiles(const Lattice &L, Ctrl *C, uint32_t g,
                                               uint32_t *nw32, uint32_t *ntiles) {
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  *nw32 = (uint32_t)((last - first + 31) / 32);
  *ntiles = (*nw32 + TW - 1) / TW;
  if ((uint64_t)(*ntiles) * L.l1p * bs_stride(TW) > L.vwords || L.tw != (uint32_t)TW) {
    if (threadIdx.x == 0) C->error = DIC_INTERNAL_BOUNDS;
    return false;
  }
  return true;
}

// Windows up to this many counted records use bs_count_direct.
constexpr uint32_t BS_DIRECT_MAX = 24576;

// Count records [lo, hi) with one warp per record: lane w reads word w of
// each of the record's rank columns from the block's column buffer (tile
// t = w / TW), ANDs them and
// popcounts; the warp sum is the record's count. Then PRUNE (tallies and
// algorithmic work are added to the caller's counters). The ranks are
// held in registers and the rank loop is unrolled (predicated on q < k) so
// that a lane's column loads, and those of its next words, are all in
// flight together. Whole warps must call this
// (grid-stride over records by warp).
template <int TW, int KRE, uint32_t UJ = 4>
__device__ __forceinline__ void bs_count_direct(const Lattice &L, Ctrl *C, uint32_t g,
                                                uint32_t lo, uint32_t hi, uint32_t nw32,
                                                uint32_t &pruned, uint32_t &solid,
                                                unsigned long long &work) {
  constexpr uint32_t ST = bs_stride(TW);
  static_assert(KRMAX == 16, "ranks are loaded as two 16-byte words");
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint32_t *__restrict__ V = vcols(L, g);
  const uint32_t l1p = L.l1p;
  for (uint64_t c = lo + (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < hi;
       c += nwarps) {
    // the record's state and all its ranks in one round of independent loads
    // (lane 0 keeps what PRUNE needs; the ranks are broadcast from the same
    // two 16-byte words)
    const uint8_t sh = L.cshape[c];
    const uint32_t k8 = L.ck[c];
    const uint4 *rk4 = reinterpret_cast<const uint4 *>(L.cranks + c * KRMAX);
    const uint4 ra = __ldg(rk4);
    const uint4 rb = KRE > 8 ? __ldg(rk4 + 1) : make_uint4(0u, 0u, 0u, 0u);
    uint32_t supp0 = 0, birth = 0;
    if (lane == 0) { supp0 = L.csupp[c]; birth = L.cbirth[c]; }
    const uint32_t k = sh == SH_NIL ? 0u : k8;
    if (k == 0) continue;  // uniform over the warp
    const uint32_t rw[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
    uint32_t r[KRE];
#pragma unroll
    for (int q = 0; q < KRE; ++q)
      r[q] = (uint32_t)q < k ? (rw[q >> 1] >> (16 * (q & 1))) & 0xFFFFu : 0u;
    // 16-byte loads: lane j takes words 4j .. 4j+3 of every rank column
    // (a tile row holds TW = 4, 8 or 16 words, so the four share a tile;
    // words past the block's rows are zero in the buffer). UJ loads per
    // rank are issued before any AND.
    const uint32_t nv = (nw32 + 3) / 4;
    uint32_t cnt = 0;
    for (uint32_t j0 = 0; j0 < nv; j0 += 32 * UJ) {
      uint4 acc[UJ];
#pragma unroll
      for (uint32_t u = 0; u < UJ; ++u) {
        const uint32_t j = j0 + 32 * u + lane;
        const uint32_t w = 4 * j;
        const uint64_t base = (uint64_t)(w / TW) * l1p;
        const uint32_t wi = w % TW;
        acc[u] = j < nv ? __ldg(reinterpret_cast<const uint4 *>(V + (base + r[0]) * ST + wi))
                        : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int q = 1; q < KRE; ++q) {
          if ((uint32_t)q < k && j < nv) {
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(V + (base + r[q]) * ST + wi));
            acc[u].x &= x.x; acc[u].y &= x.y; acc[u].z &= x.z; acc[u].w &= x.w;
          }
        }
      }
#pragma unroll
      for (uint32_t u = 0; u < UJ; ++u)
        cnt += __popc(acc[u].x) + __popc(acc[u].y) + __popc(acc[u].z) + __popc(acc[u].w);
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) {
      const uint32_t s = supp0 + cnt;
      L.csupp[c] = s;
      settle_loaded(L, C, (uint32_t)c, sh, birth, s, g, true, pruned, solid);
      work += (unsigned long long)(k + 1) * nw32;
    }
  }
}

// Count records [c0, c0+cn) of the window over the block of stop g and apply
// PRUNE (Algorithm 4) to each. Tiles of the columns stream through a cp.async double
// buffer; every thread ANDs its candidates' rank columns with 128-bit shared
// loads and popcounts. The whole CTA must call this (it synchronises).
template <int TW, int KRE, int NT>
__device__ __forceinline__ void bs_count_chunk(const Lattice &L, Ctrl *C, uint32_t g, uint32_t c0,
                                               uint32_t cn, uint32_t nw32, uint32_t ntiles,
                                               uint32_t *sm, uint32_t chunk_cap,
                                               uint32_t &pruned, uint32_t &solid,
                                               unsigned long long &work) {
  constexpr uint32_t ST = bs_stride(TW);
  constexpr int NV = TW / 4;  // 128-bit loads per rank and tile
  const uint32_t tile_words = L.l1p * ST;
  const uint32_t *V = vcols(L, g);
  uint32_t *S0 = sm;
  uint32_t *S1 = sm + tile_words;
  uint16_t *rk = reinterpret_cast<uint16_t *>(sm + 2 * tile_words);
  uint32_t *cnt = reinterpret_cast<uint32_t *>(rk + (size_t)chunk_cap * KRE);
  uint8_t *kk = reinterpret_cast<uint8_t *>(cnt + chunk_cap);
  const uint32_t tid = threadIdx.x;
  // records below `skip` (the pair cohort while the tensor path counts it)
  // already have this stop's count: only PRUNE is applied to them
  const uint32_t skip = (L.pair_end && g <= L.stop_max) ? L.pair_end : 0u;
  const bool need_tiles = c0 + cn > skip;  // uniform over the CTA
  __syncthreads();  // shared memory of the previous chunk is free
  if (need_tiles) {
    for (uint32_t o = tid * 4; o < tile_words; o += NT * 4) cp_async16(S0 + o, V + o);
    cp_async_commit();
  }
  for (uint32_t i = tid; i < cn; i += NT) {
    const uint32_t c = c0 + i;
    const uint32_t k = L.cshape[c] == SH_NIL ? 0u : (uint32_t)L.ck[c];
    kk[i] = (uint8_t)(k && c < skip ? KSKIP : k);
    cnt[i] = 0;
    if (c < skip) continue;  // counted elsewhere: no ranks needed
#pragma unroll
    for (int q = 0; q < KRE; ++q)
      rk[(size_t)i * KRE + q] = (uint32_t)q < k ? L.cranks[(uint64_t)c * KRMAX + q] : (uint16_t)0;
  }
  for (uint32_t t = 0; need_tiles && t < ntiles; ++t) {
    if (t + 1 < ntiles) {
      uint32_t *dst = ((t + 1) & 1) ? S1 : S0;
      const uint32_t *src = V + (size_t)(t + 1) * tile_words;
      for (uint32_t o = tid * 4; o < tile_words; o += NT * 4) cp_async16(dst + o, src + o);
    }
    cp_async_commit();
    cp_async_wait_1();
    __syncthreads();
    const uint32_t *S = (t & 1) ? S1 : S0;
    for (uint32_t i = tid; i < cn; i += NT) {
      const uint32_t k = kk[i];
      if (k == 0 || k == KSKIP) continue;
      const uint16_t *ri = rk + (size_t)i * KRE;
      uint4 acc[NV];
      {
        const uint4 *p = reinterpret_cast<const uint4 *>(S + (uint32_t)ri[0] * ST);
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] = p[v];
      }
      for (uint32_t q = 1; q < k; ++q) {
        const uint4 *p = reinterpret_cast<const uint4 *>(S + (uint32_t)ri[q] * ST);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const uint4 x = p[v];
          acc[v].x &= x.x; acc[v].y &= x.y; acc[v].z &= x.z; acc[v].w &= x.w;
        }
      }
      uint32_t sum = 0;
#pragma unroll
      for (int v = 0; v < NV; ++v)
        sum += __popc(acc[v].x) + __popc(acc[v].y) + __popc(acc[v].z) + __popc(acc[v].w);
      cnt[i] += sum;
    }
    __syncthreads();  // the buffer of tile t may be overwritten next
  }
  for (uint32_t i = tid; i < cn; i += NT) {
    if (!kk[i]) continue;
    const uint32_t c = c0 + i;
    if (kk[i] == KSKIP) {
      settle_record(L, C, c, L.csupp[c], g, true, pruned, solid);
      continue;
    }
    const uint32_t s = L.csupp[c] + cnt[i];
    L.csupp[c] = s;
    settle_record(L, C, c, s, g, true, pruned, solid);
    // algorithmic work: k-1 AND + POPC + ADD per 32-row word
    work += (unsigned long long)(kk[i] + 1) * nw32;
  }
}

}  // namespace dic
