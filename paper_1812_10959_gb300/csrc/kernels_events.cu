// Event-driven stop loop (single queries with every block's columns staged
// and the pair cohort counted by the all-blocks GEMM).
//
// Under Algorithm 4 a dashed circle's fate depends only on its own counts:
// after its birth at stop b it is counted over blocks b+1, b+2, ... (one per
// stop, wrapping round the database as in Algorithm 2), and at the first
// stop where its running count reaches minsup it is promoted (and then stays
// dashed until its full pass ends, when it becomes solid), or at the first
// stop where the count plus M for every block still to come falls below
// minsup it is erased. None of this depends on the rest of the lattice, so a
// cohort can be counted over its whole pass as soon as it is born, and its
// promotion and erase stops are then known in advance. The stop loop keeps
// Algorithm 2's order of decisions exactly (same promotions, erasures,
// candidates and trace rows at every stop) but only stops where something is
// promoted need MAKECANDIDATES; the trace rows of the stops in between are
// written from the per-stop tallies.
//
// One iteration of the loop is two kernels:
//   k_cohort_pass      the cohort MAKECANDIDATES produced at the prepared
//                      stop is counted over its whole pass (each record's
//                      blocks split across CTAs: AND of its items' bit
//                      columns, popc, per-block counts; the record's last
//                      part finds its promotion or erase stop and its
//                      full-pass support; future boxes go into the box set
//                      with their promotion stop). The last CTA to finish
//                      then closes that stop (trace row, CHECKFULLPASS, loop
//                      test), closes every following stop that promotes
//                      nothing, prepares the next stop that does (tallies
//                      and promoted list) and decides whether the loop
//                      graph goes on.
//   k_generate_finish  MAKECANDIDATES at the prepared stop (Lattice.events:
//                      generation only; the next cohort pass closes the
//                      stop).
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"
#include "lattice_device.cuh"

namespace dic {

constexpr int CP_THREADS = 256;

// Dynamic shared memory of k_cohort_pass: per-block counts [stop_max] and
// the record's ranks [l1] (u16).
size_t cohort_pass_smem(uint32_t stop_max, uint32_t l1) {
  return (size_t)stop_max * 4 + (((size_t)l1 * 2 + 15) & ~(size_t)15);
}

// The loop state copied into shared memory through L2 by one warp (the
// cohort pass's other CTAs have added to it with atomics since this SM last
// read it); the warp's lanes load its words in parallel.
__device__ __forceinline__ void load_ctrl_l2(const Ctrl *C, Ctrl *dst_sm) {
  static_assert(sizeof(Ctrl) % 4 == 0, "Ctrl is copied in 32-bit words");
  const uint32_t *src = reinterpret_cast<const uint32_t *>(C);
  uint32_t *dst = reinterpret_cast<uint32_t *>(dst_sm);
  for (uint32_t i = threadIdx.x & 31; i < sizeof(Ctrl) / 4; i += 32) dst[i] = __ldcg(src + i);
  __syncwarp();
}

// List record c (promoted at the stop being prepared, its box-set entry
// already made) for MAKECANDIDATES: slot, size, first two ranks and the
// hash pre-image sum of its mask.
__device__ __forceinline__ void list_promoted(const Lattice &L, Ctrl *C, uint32_t c) {
  const uint32_t k = L.ck[c];
  const uint32_t r01 = *reinterpret_cast<const uint32_t *>(L.cranks + (uint64_t)c * KRMAX);
  const uint32_t at = atomicAdd(&C->n_newbox, 1u);
  L.newbox[at] = c;
  L.newinfo[at] = (uint64_t)k | ((uint64_t)(r01 & 0xFFFFu) << 8) | ((uint64_t)(r01 >> 16) << 24);
  L.newhash[at] = mask_hash_sum(L.cmask + (uint64_t)c * L.wc, L.wc);
}

// Tallies of stop s for the trace (pairs from the precomputed pair events,
// longer records from the cohort passes) and whether s promotes anything.
struct StopTally {
  uint32_t promoted, pruned, solid, eb;
};
__device__ __forceinline__ StopTally stop_tally(const Lattice &L, uint32_t s) {
  StopTally t;
  const bool pl = L.pair_events && s <= L.stop_max;
  const uint32_t np = pl ? L.ev_off[s + 1] - L.ev_off[s] : 0u;
  t.eb = L.eh_box[s];
  t.promoted = np + t.eb;
  t.pruned = (pl ? L.ev_pruned[s] : 0u) + L.eh_pruned[s];
  t.solid = ((L.pair_events && s == L.stop_max) ? L.ev_pruned[0] : 0u) + L.eh_solid[s];
  return t;
}

// Warp 0 of the last CTA: close the stop MAKECANDIDATES just ran at (if one
// is pending), then every following stop that promotes nothing (at most
// `budget`), and prepare the stop the walk ends on: its tallies go to the
// loop state and (when it promotes something) the whole CTA lists its
// promoted records afterwards. Lanes load the tallies of 32 stops at once;
// lane 0 holds the loop state and closes the stops in order. The results go
// to the caller's shared words: a stop prepared with promotions (s_act), its
// number, its listed count, the window of longer records, and whether the
// loop graph goes on (s_more).
__device__ void ev_advance(const Lattice &L, Ctrl *C, uint32_t budget, uint32_t *s_act,
                           uint32_t *s_s, uint32_t *s_eb, uint32_t *s_lo, uint32_t *s_tail,
                           uint32_t *s_more) {
  __shared__ Ctrl s_ctrl;
  const uint32_t lane = threadIdx.x & 31;
  load_ctrl_l2(C, &s_ctrl);
  Ctrl c = s_ctrl;  // meaningful in lane 0 (the others follow its decisions)
  if (lane == 0 && c.ev_iter < L.ehcap) L.ev_work[c.ev_iter] = c.work;
  if (lane == 0 && c.ev_pending) {
    // the stop MAKECANDIDATES ran at: its candidate count is final
    if (c.n_trace >= L.tcap) {
      C->stall = ST_TRACE;
      c.stall = ST_TRACE;
    } else {
      finish_stop_with(L, C, c);
    }
  }
  uint32_t stop_walk = __shfl_sync(0xffffffffu, (c.done || c.error || c.stall) ? 1u : 0u, 0);
  uint32_t act = 0, prepared = 0, it = 0;
  while (!stop_walk) {
    const uint32_t s0 = __shfl_sync(0xffffffffu, c.step, 0);
    const uint32_t s = s0 + lane;
    StopTally t = {0, 0, 0, 0};
    const bool in = s + 1 < L.ehcap;
    if (in) t = stop_tally(L, s);
    for (uint32_t i = 0; i < 32; ++i) {
      const bool in_i = __shfl_sync(0xffffffffu, in ? 1u : 0u, i) != 0;
      const uint32_t pro = __shfl_sync(0xffffffffu, t.promoted, i);
      const uint32_t pru = __shfl_sync(0xffffffffu, t.pruned, i);
      const uint32_t sol = __shfl_sync(0xffffffffu, t.solid, i);
      const uint32_t eb = __shfl_sync(0xffffffffu, t.eb, i);
      const uint32_t room = __shfl_sync(0xffffffffu, c.n_trace + 1 < L.tcap ? 1u : 0u, 0);
      if (!in_i || !room) {
        if (lane == 0) C->stall = ST_TRACE;  // the host grows the trace and the tallies
        stop_walk = 1;
        break;
      }
      if (pro > 0 || it >= budget) {
        if (lane == 0) {
          C->n_pruned = pru;
          C->n_solid = sol;
          C->n_newbox = 0;
          C->gen_ticket = 0;
          *s_s = s0 + i;
          *s_eb = eb;
          *s_lo = c.head > L.pair_end ? c.head : L.pair_end;
          *s_tail = c.tail;
        }
        act = pro > 0 ? 1u : 0u;
        prepared = 1;
        stop_walk = 1;
        break;
      }
      if (lane == 0) {
        c.n_pruned = pru;
        c.n_solid = sol;
        c.n_newbox = 0;
        c.gen_ticket = 0;
        finish_stop_with(L, C, c);
      }
      ++it;
      if (__shfl_sync(0xffffffffu, (c.done || c.error) ? 1u : 0u, 0)) {
        stop_walk = 1;
        break;
      }
    }
  }
  if (lane == 0) {
    C->ev_pending = prepared;
    C->ev_iter = c.ev_iter + 1;
    *s_act = act;
    // the loop graph goes on while a stop is prepared and the iteration
    // limit is not reached
    *s_more = prepared && c.ev_iter + 1 < c.ev_limit ? 1u : 0u;
  }
  __syncwarp();
}

// Count the items of rank list s_rank[0..k) over blocks [b0, b1) of the pass
// into s_cnt[block - b0]: work items (block, 128-row group j), U per thread
// at a time; the 16-byte words of four ranks are loaded for all U items
// before any AND (a rank index past k repeats rank 0: ANDing a column twice
// changes nothing), then each item's popc goes to its block's counter.
// Threads tid = 0..nt-1 of the caller's group (the CTA, or one warp) share
// the work items.
template <int TW>
__device__ __forceinline__ void cp_count(const Lattice &L, const uint16_t *s_rank, uint32_t k,
                                         uint32_t b0, uint32_t b1, uint32_t nvmax,
                                         uint32_t *s_cnt, uint32_t tid, uint32_t nt) {
  constexpr uint32_t ST = bs_stride(TW);
  constexpr int U = 4;
  const uint32_t l1p = L.l1p;
  const uint64_t items = (uint64_t)(b1 - b0) * nvmax;
  for (uint64_t it0 = tid; it0 < items; it0 += (uint64_t)nt * U) {
    const uint32_t *Vu[U];
    uint32_t blk[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t it = it0 + (uint64_t)u * nt;
      const uint64_t itc = it < items ? it : 0;  // item 0 stands in (result unused)
      const uint32_t a = (uint32_t)(itc / nvmax), j = (uint32_t)(itc % nvmax);
      const uint32_t w = 4 * j;
      blk[u] = it < items ? a : ~0u;
      Vu[u] = L.V + (uint64_t)(b0 + a) * L.vwords + (uint64_t)(w / TW) * l1p * ST + (w % TW);
    }
    uint4 acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) acc[u] = make_uint4(~0u, ~0u, ~0u, ~0u);
    for (uint32_t q0 = 0; q0 < k; q0 += 4) {
      uint4 x[4][U];
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        const uint32_t q = q0 + qq;
        const uint64_t r = s_rank[q < k ? q : 0];
#pragma unroll
        for (int u = 0; u < U; ++u) x[qq][u] = __ldg(reinterpret_cast<const uint4 *>(Vu[u] + r * ST));
      }
#pragma unroll
      for (int qq = 0; qq < 4; ++qq)
#pragma unroll
        for (int u = 0; u < U; ++u) {
          acc[u].x &= x[qq][u].x; acc[u].y &= x[qq][u].y;
          acc[u].z &= x[qq][u].z; acc[u].w &= x[qq][u].w;
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (blk[u] == ~0u) continue;
      const uint32_t p = __popc(acc[u].x) + __popc(acc[u].y) + __popc(acc[u].z) + __popc(acc[u].w);
      if (p) atomicAdd(&s_cnt[blk[u]], p);
    }
  }
}

// Warp 0: record c's event from its per-block counts cnt[0..S) (block a =
// cnt[a]; shared or global memory) over the ages 1..S in stop order (the
// block of stop g + a is (g + a - 1) mod S), and its updates.
__device__ __forceinline__ void cp_events(const Lattice &L, Ctrl *C, uint32_t c, uint32_t g,
                                          const uint32_t *cnt, bool global_cnt) {
  const uint32_t lane = threadIdx.x & 31, S = L.stop_max;
  auto ld = [&](uint32_t a) -> uint32_t { return global_cnt ? __ldcg(cnt + a) : cnt[a]; };
  uint64_t total = 0;
  for (uint32_t a = lane; a < S; a += 32) total += ld(a);
  for (int o = 16; o > 0; o >>= 1) total += __shfl_xor_sync(0xffffffffu, total, o);
  uint64_t carry = 0;
  uint32_t ev_age = 0, ev_promote = 0;
  uint64_t ev_cum = 0;
  for (uint32_t base = 0; base < S; base += 32) {
    const uint32_t age = base + lane + 1;
    const uint32_t v = age <= S ? ld((g + age - 1) % S) : 0u;
    uint64_t cum = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, cum, o);
      if (lane >= (uint32_t)o) cum += y;
    }
    cum += carry;
    const bool prom = age <= S && cum >= L.minsup;
    const bool drop = age <= S && cum + L.M * (uint64_t)(S - age) < (uint64_t)L.minsup;
    const uint32_t bal = __ballot_sync(0xffffffffu, prom || drop);
    if (bal) {
      const int src = __ffs(bal) - 1;
      ev_age = base + src + 1;
      ev_promote = __shfl_sync(0xffffffffu, prom ? 1u : 0u, src);
      ev_cum = __shfl_sync(0xffffffffu, cum, src);
      break;
    }
    carry = __shfl_sync(0xffffffffu, cum, 31);
  }
  if (lane != 0) return;
  // every record meets one of the two by age S (there the bound is its full
  // support), so ev_age >= 1
  const uint32_t p = g + ev_age;
  if (ev_age == 0 || p + 1 >= L.ehcap || g + S + 1 >= L.ehcap) {
    C->error = DIC_INTERNAL_BOUNDS;
  } else if (ev_promote) {
    L.csupp[c] = (uint32_t)total;
    L.cshape[c] = SH_BOX;
    L.cpromo[c] = p;
    box_insert(L, c, mask_hash_sum(L.cmask + (uint64_t)c * L.wc, L.wc));
    const uint32_t i = atomicAdd(&L.eh_box[p], 1u);
    if (i < EV_LIST) L.eb_list[(uint64_t)p * EV_LIST + i] = c;
    atomicAdd(&L.eh_solid[g + S], 1u);
  } else {
    L.csupp[c] = (uint32_t)ev_cum;
    L.cshape[c] = SH_NIL;
    atomicAdd(&L.eh_pruned[p], 1u);
  }
}

template <int TW>
__global__ void __launch_bounds__(CP_THREADS, 2) k_cohort_pass(Lattice L, uint32_t budget,
                                                            uint32_t use_cond,
                                                            unsigned long long cond) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) uint8_t cps[];
  uint32_t *s_cnt = reinterpret_cast<uint32_t *>(cps);
  uint16_t *s_rank = reinterpret_cast<uint16_t *>(cps + (size_t)L.stop_max * 4);
  __shared__ uint32_t s_go, s_lo, s_n, s_birth, s_last, s_k, s_rlast;
  __shared__ uint32_t s_act, s_s, s_eb, s_wlo, s_tail, s_more;
  Ctrl *C = L.ctrl;
  if (threadIdx.x == 0) {
    const uint32_t stall = C->stall, done = C->done, err = C->error;
    const uint32_t hash_used = C->hash_used, n_live = C->n_live;
    const uint32_t pending = C->ev_pending;
    const uint32_t n_gen = (uint32_t)C->gen_ticket;
    // the cohort MAKECANDIDATES emitted at the pending stop
    s_lo = C->tail;
    s_n = pending ? n_gen : 0u;
    s_birth = C->step;
    uint32_t go = !stall && !done && !err;
    // room in the box set for every live record and the new cohort (whose
    // future boxes are inserted now); decided alike by every CTA from values
    // no CTA of this launch changes
    if (go && (uint64_t)(hash_used + n_live + s_n) * 2 > L.hcap) {
      go = 0;
      if (blockIdx.x == 0) C->stall = ST_HASH_EV;
    }
    if (go && (uint64_t)s_lo + s_n > L.cap) go = 0;  // (a generation stall is pending)
    s_go = go;
    if (!go && use_cond && blockIdx.x == 0) cudaGraphSetConditional(cond, 0);
  }
  __syncthreads();
  if (!s_go) return;
  const uint32_t g = s_birth, S = L.stop_max, n = s_n;
  const uint64_t blockmax = L.M < L.n ? L.M : L.n;
  const uint32_t nw32max = (uint32_t)((blockmax + 31) / 32);
  const uint32_t nvmax = (nw32max + 3) / 4;
  // 32-row words of the whole pass (the last block may be short)
  const uint64_t last_rows = L.n - (uint64_t)(S - 1) * L.M;
  const uint64_t pass_words = (uint64_t)(S - 1) * nw32max + (last_rows + 31) / 32;
  // each record's blocks in R contiguous parts (R > 1 when the cohort is
  // small enough for the per-record scratch counts)
  uint32_t R = 1;
  if (n && n <= L.cp_records) {
    R = gridDim.x / n;  // one unit per CTA
    R = R < 1 ? 1 : (R > S ? S : R);
  }
  unsigned long long work = 0;
  const uint64_t units = (uint64_t)n * R;
  for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const uint32_t ci = (uint32_t)(u / R), part = (uint32_t)(u % R);
    const uint32_t c = s_lo + ci;
    const uint32_t b0 = (uint32_t)((uint64_t)part * S / R);
    const uint32_t b1 = (uint32_t)((uint64_t)(part + 1) * S / R);
    // the record's ranks (from its mask when it has more than KRMAX items)
    if (threadIdx.x == 0) {
      // size and all stored ranks in one round of loads
      uint32_t k = L.ck[c];
      const uint4 *rk4 = reinterpret_cast<const uint4 *>(L.cranks + (uint64_t)c * KRMAX);
      const uint4 ra = rk4[0], rb = rk4[1];
      if (k <= (uint32_t)KRMAX) {
        const uint32_t rw[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
        for (uint32_t q = 0; q < k; ++q) s_rank[q] = (uint16_t)(rw[q >> 1] >> (16 * (q & 1)));
      } else {
        k = 0;
        for (uint32_t i = 0; i < L.wc; ++i)
          for (uint64_t x = L.cmask[(uint64_t)c * L.wc + i]; x; x &= x - 1)
            if (k < L.l1) s_rank[k++] = (uint16_t)(i * 64 + __ffsll((long long)x) - 1);
      }
      s_k = k;
      s_rlast = 0;
    }
    for (uint32_t a = threadIdx.x; a < b1 - b0; a += blockDim.x) s_cnt[a] = 0;
    __syncthreads();
    const uint32_t k = s_k;
    if (k) cp_count<TW>(L, s_rank, k, b0, b1, nvmax, s_cnt, threadIdx.x, blockDim.x);
    __syncthreads();
    if (R == 1) {
      if (threadIdx.x < 32) cp_events(L, C, c, g, s_cnt, false);
    } else {
      // this part's counts to the record's scratch row; the record's last
      // part to finish decides its events from the whole row
      uint32_t *row = L.cp_cnt + (uint64_t)ci * S;
      for (uint32_t a = threadIdx.x; a < b1 - b0; a += blockDim.x) row[b0 + a] = s_cnt[a];
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t t = atomicAdd(&L.cp_tick[ci], 1u);
        s_rlast = t == R - 1 ? 1u : 0u;
        if (s_rlast) {
          __threadfence();
          L.cp_tick[ci] = 0;  // ready for the next cohort
        }
      }
      __syncthreads();
      if (s_rlast && threadIdx.x < 32) cp_events(L, C, c, g, row, true);
    }
    if (threadIdx.x == 0 && (R == 1 || s_rlast)) work += (unsigned long long)(k + 1) * pass_words;
    __syncthreads();  // shared counts and ranks are reused by the next unit
  }
  // the last CTA to finish closes the pending stop and advances the loop
  if (threadIdx.x == 0) {
    if (work) atomicAdd(&C->work, work);
    __threadfence();
    const uint32_t t = atomicAdd(&C->ev_ticket, 1u);
    s_last = t == gridDim.x - 1 ? 1u : 0u;
    if (s_last) {
      __threadfence();
      C->ev_ticket = 0;
    }
    s_act = 0;
    s_more = 0;
  }
  __syncthreads();
  if (!s_last) return;
  if (threadIdx.x < 32) ev_advance(L, C, budget, &s_act, &s_s, &s_eb, &s_wlo, &s_tail, &s_more);
  __syncthreads();
  if (threadIdx.x == 0 && use_cond && !s_more) cudaGraphSetConditional(cond, 0);
  if (!s_act) return;
  // the promoted list of the prepared stop: its pairs (precomputed), then
  // its longer records
  const uint32_t s = s_s;
  if (L.pair_events && s <= L.stop_max) {
    const uint32_t e0 = L.ev_off[s], e1 = L.ev_off[s + 1];
    for (uint32_t i = e0 + threadIdx.x; i < e1; i += blockDim.x)
      promote_record(L, C, L.ev_list[i], s, false);
  }
  const uint32_t eb = s_eb;
  if (eb <= EV_LIST) {
    for (uint32_t i = threadIdx.x; i < eb; i += blockDim.x)
      list_promoted(L, C, L.eb_list[(uint64_t)s * EV_LIST + i]);
  } else {  // more than the per-stop list holds: find them in the window
    for (uint32_t c = s_wlo + threadIdx.x; c < s_tail; c += blockDim.x)
      if (L.cpromo[c] == s) list_promoted(L, C, c);
  }
}

// Window pass (the hand-over from the per-stop loop at stop `step`) over the
// live records c of [lo, hi). A record has been counted over ages 1..a0
// (a0 = step - 1 - birth blocks) and holds that count in csupp; its blocks
// of ages a0 + 1..S (a cyclic range of block indices) are counted now, in
// work units of up to `cb` blocks shared out among all warps: a record born
// just before the hand-over has nearly a whole pass left, one near the end
// of its pass a block or two, and units keep the warps evenly loaded. A
// unit's per-block counts go to the record's scratch row rows[c - lo][block];
// the warp that finishes the record's last unit (ticket tick[c - lo]) scans
// the row in stop order and continues Algorithm 4 from there: a circle's
// promotion or erase stop, a box's full-pass support; the tallies and
// box-set entries are those of the cohort pass. Each warp first looks at 32
// units at once (a lane each: the record's shape and birth) and counts only
// those that are live.
constexpr uint32_t WP_CBMAX = 64;  // blocks per unit at most
constexpr uint32_t WP_WARPS = CP_THREADS / 32;

template <int TW>
__global__ void __launch_bounds__(CP_THREADS, 2)
    k_window_pass(Lattice L, uint32_t lo, uint32_t hi, uint32_t step, uint32_t cb,
                  uint32_t rank_stride, uint32_t *__restrict__ rows,
                  uint32_t *__restrict__ tick) {
  extern __shared__ __align__(16) uint8_t cps[];
  __shared__ uint32_t s_cnt_all[WP_WARPS][WP_CBMAX];
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  Ctrl *C = L.ctrl;
  const uint32_t S = L.stop_max, P = (S + cb - 1) / cb;
  uint32_t *s_cnt = s_cnt_all[warp];
  uint16_t *s_rank = reinterpret_cast<uint16_t *>(cps) + (size_t)warp * rank_stride;
  const uint64_t blockmax = L.M < L.n ? L.M : L.n;
  const uint32_t nw32max = (uint32_t)((blockmax + 31) / 32);
  const uint32_t nvmax = (nw32max + 3) / 4;
  const uint64_t last_rows = L.n - (uint64_t)(S - 1) * L.M;
  const uint32_t last_w32 = (uint32_t)((last_rows + 31) / 32);
  const uint64_t units = (uint64_t)(hi - lo) * P;
  const uint64_t gw = (uint64_t)blockIdx.x * nwarp + warp, nw = (uint64_t)gridDim.x * nwarp;
  unsigned long long work = 0;
  for (uint64_t r0 = 0; gw + r0 * nw < units; r0 += 32) {
    // lane i looks at unit gw + (r0 + i) * nw
    const uint64_t u = gw + (r0 + lane) * nw;
    uint32_t ci = 0, part = 0, birth = 0, sh = SH_NIL;
    bool live = false;
    if (u < units) {
      ci = (uint32_t)(u / P);
      part = (uint32_t)(u % P);
      sh = L.cshape[lo + ci];
      birth = L.cbirth[lo + ci];
      const uint32_t a0 = step - 1 - birth;
      live = sh != SH_NIL && a0 < S && part * cb < S - a0;
    }
    for (uint32_t bal = __ballot_sync(0xffffffffu, live); bal; bal &= bal - 1) {
      const int src = __ffs(bal) - 1;
      const uint32_t uci = __shfl_sync(0xffffffffu, ci, src);
      const uint32_t upart = __shfl_sync(0xffffffffu, part, src);
      const uint32_t ub = __shfl_sync(0xffffffffu, birth, src);
      const uint32_t ush = __shfl_sync(0xffffffffu, sh, src);
      const uint32_t c = lo + uci, a0 = step - 1 - ub, len = S - a0;
      const uint32_t nparts = (len + cb - 1) / cb, off = upart * cb;
      const uint32_t cnt = len - off < cb ? len - off : cb;
      uint32_t k = 0;
      if (lane == 0) k = L.ck[c];
      k = __shfl_sync(0xffffffffu, k, 0);
      if (k <= (uint32_t)KRMAX) {
        if (lane < k) s_rank[lane] = L.cranks[(uint64_t)c * KRMAX + lane];
      } else {
        if (lane == 0) {
          k = 0;
          for (uint32_t i = 0; i < L.wc; ++i)
            for (uint64_t x = L.cmask[(uint64_t)c * L.wc + i]; x; x &= x - 1)
              if (k < L.l1) s_rank[k++] = (uint16_t)(i * 64 + __ffsll((long long)x) - 1);
        }
        k = __shfl_sync(0xffffffffu, k, 0);
      }
      for (uint32_t j = lane; j < cb; j += 32) s_cnt[j] = 0;
      __syncwarp();
      // this unit's blocks: cnt of them from (birth + a0 + off) mod S on
      const uint32_t x = (ub + a0 + off) % S;
      const uint32_t e1 = x + cnt < S ? x + cnt : S;
      if (k) {
        cp_count<TW>(L, s_rank, k, x, e1, nvmax, s_cnt, lane, 32);
        if (x + cnt > S) cp_count<TW>(L, s_rank, k, 0, x + cnt - S, nvmax, s_cnt + (S - x), lane, 32);
      }
      __syncwarp();
      uint32_t *row = rows + (uint64_t)uci * S;
      for (uint32_t j = lane; j < cnt; j += 32) row[(x + j) % S] = s_cnt[j];
      __syncwarp();
      uint32_t last = 0;
      if (lane == 0) {
        __threadfence();
        const uint32_t t = atomicAdd(&tick[uci], 1u);
        last = t == nparts - 1 ? 1u : 0u;
        if (last) {
          __threadfence();
          tick[uci] = 0;  // ready for the next batch
        }
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last) {
        uint32_t cum0 = 0;
        if (lane == 0) cum0 = L.csupp[c];
        cum0 = __shfl_sync(0xffffffffu, cum0, 0);
        uint64_t rest = 0;
        for (uint32_t age = a0 + 1 + lane; age <= S; age += 32)
          rest += __ldcg(row + (ub + age - 1) % S);
        for (int o = 16; o > 0; o >>= 1) rest += __shfl_xor_sync(0xffffffffu, rest, o);
        const uint64_t total = cum0 + rest;
        uint32_t ev_age = 0, ev_promote = 0;
        uint64_t ev_cum = 0;
        if (ush == SH_CIRCLE) {
          uint64_t carry = cum0;
          for (uint32_t base = a0; base < S; base += 32) {
            const uint32_t age = base + lane + 1;
            const uint32_t v = age <= S ? __ldcg(row + (ub + age - 1) % S) : 0u;
            uint64_t cum = v;
            for (int o = 1; o < 32; o <<= 1) {
              const uint64_t y = __shfl_up_sync(0xffffffffu, cum, o);
              if (lane >= (uint32_t)o) cum += y;
            }
            cum += carry;
            const bool prom = age <= S && cum >= L.minsup;
            const bool drop = age <= S && cum + L.M * (uint64_t)(S - age) < (uint64_t)L.minsup;
            const uint32_t b2 = __ballot_sync(0xffffffffu, prom || drop);
            if (b2) {
              const int s2 = __ffs(b2) - 1;
              ev_age = base + s2 + 1;
              ev_promote = __shfl_sync(0xffffffffu, prom ? 1u : 0u, s2);
              ev_cum = __shfl_sync(0xffffffffu, cum, s2);
              break;
            }
            carry = __shfl_sync(0xffffffffu, cum, 31);
          }
        }
        if (lane == 0) {
          const uint32_t solid_at = ub + S;
          if (solid_at + 1 >= L.ehcap || (ush == SH_CIRCLE && ev_age == 0)) {
            C->error = DIC_INTERNAL_BOUNDS;
          } else if (ush == SH_BOX) {  // promoted earlier: the rest of its pass
            L.csupp[c] = (uint32_t)total;
            atomicAdd(&L.eh_solid[solid_at], 1u);
          } else if (ev_promote) {
            const uint32_t p = ub + ev_age;
            L.csupp[c] = (uint32_t)total;
            L.cshape[c] = SH_BOX;
            L.cpromo[c] = p;
            box_insert(L, c, mask_hash_sum(L.cmask + (uint64_t)c * L.wc, L.wc));
            const uint32_t i = atomicAdd(&L.eh_box[p], 1u);
            if (i < EV_LIST) L.eb_list[(uint64_t)p * EV_LIST + i] = c;
            atomicAdd(&L.eh_solid[solid_at], 1u);
          } else {
            const uint32_t p = ub + ev_age;
            L.csupp[c] = (uint32_t)ev_cum;
            L.cshape[c] = SH_NIL;
            atomicAdd(&L.eh_pruned[p], 1u);
          }
          // 32-row words of the blocks counted now: len full blocks, the
          // last block of the pass (index S - 1) shorter if among them
          const uint32_t x0 = (ub + a0) % S;
          const bool has_last = (S - 1 + S - x0) % S < len;
          const uint64_t words =
              (uint64_t)len * nw32max - (has_last ? (uint64_t)(nw32max - last_w32) : 0ull);
          work += (unsigned long long)(k + 1) * words;
        }
      }
      __syncwarp();  // the warp's shared counts and ranks are reused next
    }
  }
  if (lane == 0 && work) atomicAdd(&C->work, work);
}

// Scratch of one window-pass launch: per-block count rows and tickets of
// up to this many records (the host launches one batch after another).
uint32_t window_pass_batch(uint32_t stop_max, uint32_t nrec) {
  const uint64_t per = std::max<uint64_t>(1, (256ull << 20) / ((uint64_t)stop_max * 4));
  return (uint32_t)std::min<uint64_t>(nrec, per);
}

template <int TW>
static cudaError_t go_wp(Lattice L, uint32_t lo, uint32_t hi, uint32_t step, uint32_t *rows,
                         uint32_t *tick, int grid, cudaStream_t s) {
  const uint64_t blockmax = L.M < L.n ? L.M : L.n;
  const uint32_t nvmax = (uint32_t)(((blockmax + 31) / 32 + 3) / 4);
  // about 512 work items (four 32-row words each) per unit
  const uint32_t cb = std::max<uint32_t>(1, std::min<uint32_t>(WP_CBMAX, 512 / nvmax));
  // each warp's ranks (a record's items, from its mask past KRMAX): as many
  // warps per CTA, up to eight, as fit 96 KiB
  const uint32_t rank_stride = (L.l1 + 7) & ~7u;
  uint32_t nwarp = (uint32_t)((96u << 10) / ((size_t)rank_stride * 2));
  nwarp = std::max<uint32_t>(1, std::min<uint32_t>(WP_WARPS, nwarp));
  const size_t smem = (size_t)nwarp * rank_stride * 2;
  cudaError_t e = cudaFuncSetAttribute(k_window_pass<TW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_window_pass<TW><<<grid, nwarp * 32, smem, s>>>(L, lo, hi, step, cb, rank_stride, rows, tick);
  return cudaGetLastError();
}

cudaError_t launch_window_pass(Lattice L, uint32_t lo, uint32_t hi, uint32_t step,
                               uint32_t *rows, uint32_t *tick, int grid, cudaStream_t s) {
  if (lo >= hi) return cudaSuccess;
  switch (L.tw) {
    case 16: return go_wp<16>(L, lo, hi, step, rows, tick, grid, s);
    case 8: return go_wp<8>(L, lo, hi, step, rows, tick, grid, s);
    case 4: return go_wp<4>(L, lo, hi, step, rows, tick, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

__global__ void k_set_ev_limit(Ctrl *C, uint32_t limit) { C->ev_limit = limit; }

cudaError_t launch_set_ev_limit(Ctrl *C, uint32_t limit, cudaStream_t s) {
  k_set_ev_limit<<<1, 1, 0, s>>>(C, limit);
  return cudaGetLastError();
}

template <int TW>
static cudaError_t go_cp(Lattice L, int grid, uint32_t budget, uint32_t use_cond,
                         unsigned long long cond, cudaStream_t s) {
  const size_t smem = cohort_pass_smem(L.stop_max, L.l1);
  cudaError_t e = cudaFuncSetAttribute(k_cohort_pass<TW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_k(k_cohort_pass<TW>, grid, CP_THREADS, smem, s, L, budget, use_cond, cond);
}

cudaError_t launch_cohort_pass(Lattice L, int grid, uint32_t budget, uint32_t use_cond,
                               unsigned long long cond, cudaStream_t s) {
  switch (L.tw) {
    case 16: return go_cp<16>(L, grid, budget, use_cond, cond, s);
    case 8: return go_cp<8>(L, grid, budget, use_cond, cond, s);
    case 4: return go_cp<4>(L, grid, budget, use_cond, cond, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace dic
