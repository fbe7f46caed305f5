// Internal declarations of the DIC library (device lattice layout, kernel
// launchers). Not part of the public ABI (include/dic.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dic {

// Shape of an itemset record (Section 4.1): NIL = erased, CIRCLE = suspected
// infrequent, BOX = frequent. Dashed vs solid is positional: a record is
// dashed while it lies in the candidate window [head, tail).
enum Shape : uint8_t { SH_NIL = 0, SH_CIRCLE = 1, SH_BOX = 2 };

// Capacity shortfalls detected on the device. A kernel that detects one
// changes nothing, sets `stall`, and every later kernel returns at once; the
// host grows the buffer and re-runs the step from the phase named here.
// ST_HASH: the box set is too full for this stop's insertions (raised by
// the insert kernel, or by a count kernel that inserts in its epilogue, which
// then resumes at PH_COUNT: ST_HASH_COUNT).
// ST_HASH_EV: the box set has no room for a new cohort's future boxes (the
// event-driven loop's cohort pass; it resumes there). ST_TRACE: the trace or
// the per-stop tallies are full (the event-driven advance).
enum Stall : uint32_t {
  ST_NONE = 0, ST_WIDTH = 1, ST_HASH = 2, ST_CAND = 3, ST_HASH_COUNT = 4, ST_HASH_EV = 5,
  ST_TRACE = 6
};
enum Phase : int { PH_COUNT = 0, PH_PROMOTE = 1, PH_HASH = 2, PH_GEN = 3 };

constexpr int TRACE_COLS = 9;
// Ctrl.error value recorded by a kernel whose own bounds check caught an
// index outside a buffer (an internal sizing error); the access is skipped.
constexpr uint32_t DIC_INTERNAL_BOUNDS = 100;
// Ranks kept per candidate record for the BITSLICE count path; itemsets with
// more items are counted by the ROWS path.
constexpr int KRMAX = 16;

// Device-resident loop state of Algorithm 2 (one per query).
struct Ctrl {
  uint32_t step;       // global stop counter g of the next stop to run (1-based)
  uint32_t done;       // 1 once DASHED is empty
  uint32_t stall;      // Stall
  uint32_t error;      // dic_status of a device-side failure (0 = none)
  uint32_t head;       // candidate window [head, tail) = DASHED (plus erased holes)
  uint32_t tail;
  uint32_t n_live;     // |DASHED|
  uint32_t n_newbox;   // promotions at this stop
  uint32_t n_pruned;   // circles erased by the bound at this stop
  uint32_t n_solid;    // records reaching a full pass at this stop
  // low 32 bits: candidates emitted at this stop (their record slots are
  // tail + 0, 1, ..., slots past the capacity included); high 32 bits: CTAs
  // of the generate kernel that have finished (its last-block ticket). One
  // word, so the last CTA's ticket returns the final count.
  unsigned long long gen_ticket;
  uint32_t gen_tail0;  // tail before this stop's generation
  uint32_t cohort_head;
  uint32_t n_cohorts;
  uint32_t hash_used;  // occupied hash slots
  uint32_t max_k;      // largest itemset size ever placed in DASHED
  uint32_t n_trace;
  uint32_t last_birth;   // creation stop of the newest cohort
  uint32_t solo;         // 1: the batched kernels leave this query alone
  uint32_t head_birth;   // creation stop of the oldest cohort in the window
  // pair events of stop ev_stop[s] in slot s = stop % 2 (set one stop ahead
  // by the count kernel, for stop 1 by the event build; the slot a stop
  // reads is never the one its own count kernel writes): first and end
  // index into ev_list and the pairs dropped at that stop
  uint32_t ev_stop[2];
  uint32_t ev_next[6];
  unsigned long long tests;  // candidate-transaction tests so far
  unsigned long long work;   // algorithmic integer ops of the count kernels
  unsigned long long gram_rows;  // block rows whose pair cohort the GEMM counted
  // event-driven loop (Lattice.events): CTAs of the cohort pass that have
  // finished; iterations (cohort pass + generate) completed; the loop graph
  // ends once ev_iter reaches ev_limit
  uint32_t ev_ticket;
  uint32_t ev_iter;
  uint32_t ev_limit;
  // 1 while a stop is prepared (tallies and promoted list) and awaits
  // MAKECANDIDATES and its close in the next cohort pass
  uint32_t ev_pending;
  // the last stop that promoted anything (the host's test for handing the
  // rest of the loop to the event-driven form)
  uint32_t last_promo;
};

__host__ __device__ inline uint32_t n_gen_of(const Ctrl &c) { return (uint32_t)c.gen_ticket; }

// Add per-thread PRUNE tallies and count work of one CTA to the loop state
// with at most one atomic per field (every thread of the CTA must call; the
// same address taken by every warp of a launch serialises at L2).
__device__ __forceinline__ void block_add_tallies(Ctrl *C, uint32_t pruned, uint32_t solid,
                                                  unsigned long long work) {
  __shared__ uint32_t s_pr[32], s_so[32];
  __shared__ unsigned long long s_wk[32];
  const uint32_t w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  pruned = __reduce_add_sync(0xffffffffu, pruned);
  solid = __reduce_add_sync(0xffffffffu, solid);
  for (int o = 16; o > 0; o >>= 1) work += __shfl_xor_sync(0xffffffffu, work, o);
  __syncthreads();  // the arrays may hold a previous call's sums
  if (lane == 0) { s_pr[w] = pruned; s_so[w] = solid; s_wk[w] = work; }
  __syncthreads();
  if (w == 0) {
    const bool in = lane < (blockDim.x >> 5);
    pruned = __reduce_add_sync(0xffffffffu, in ? s_pr[lane] : 0u);
    solid = __reduce_add_sync(0xffffffffu, in ? s_so[lane] : 0u);
    work = in ? s_wk[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) work += __shfl_xor_sync(0xffffffffu, work, o);
    if (lane == 0) {
      if (pruned) atomicAdd(&C->n_pruned, pruned);
      if (solid) atomicAdd(&C->n_solid, solid);
      if (work) atomicAdd(&C->work, work);
    }
  }
}

// Add a per-thread amount to a 64-bit counter with one atomic per warp.
__device__ __forceinline__ void warp_add_u64(unsigned long long *dst, unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// Everything a stop's kernels touch, passed by value.
struct Lattice {
  Ctrl *ctrl;
  // candidate records, append-only; [0, head) are solid, [head, tail) dashed
  uint64_t *cmask;     // [cap][wc] compact-rank bitmaps
  uint32_t *csupp;     // [cap]
  uint32_t *cbirth;    // [cap] global stop at which the record was created
  uint8_t *cshape;     // [cap]
  uint8_t *ck;         // [cap] itemset size (saturates at 255)
  uint16_t *cranks;    // [cap][KRMAX] ascending ranks (first KRMAX of them)
  uint32_t *newbox;    // [cap] records promoted at this stop
  uint64_t *newinfo;   // [cap] their size | first rank << 8 | second rank << 24
  uint64_t *newhash;   // [cap] hash pre-image sums of those records
  uint32_t *cpromo;    // [cap] stop at which a box was promoted; ~0 while
                       // the record is not a box (set at its creation)
  uint32_t cap;
  // box set: open addressing over record indices (slot = index + 1, 0 =
  // empty); keys are the records' masks, values their promotion stops
  uint32_t *hslot;     // [hcap]
  uint32_t hcap;       // power of two
  // cohorts (records created at one stop are contiguous)
  uint32_t *cohort_start;
  uint32_t *cohort_birth;
  unsigned long long *trace;  // [tcap][TRACE_COLS]
  unsigned long long *trace_work;  // [tcap] Ctrl.work after each stop's count
  uint32_t tcap;
  // the problem
  const uint64_t *rows;  // compact rows [n][wc]
  uint64_t n;
  uint64_t M;
  uint32_t stop_max;
  uint32_t minsup;
  uint32_t wc;         // words per compact row / mask
  uint32_t l1;         // frequent items (compact ranks 0..l1-1)
  // BITSLICE column buffer (nullptr when that path is not set up)
  uint32_t *V;
  uint64_t vwords;
  uint32_t tw;
  uint32_t l1p;
  // records [0, pair_end) (the pair cohort) are counted by the tensor path
  // while it is live; 0 when that path is off
  uint32_t pair_end;
  // 1: V holds two column buffers of vwords words each, stop g's block in
  // buffer g % 2 (the next block is transposed while this one is counted)
  uint32_t vdouble;
  // 1: records [0, l1(l1-1)/2) are all pairs of ranks in lexicographic order
  // (the first pass's pair join); 0 for classic DIC, whose pairs are
  // generated one by one
  uint32_t pairs_lex;
  // 1: V holds the columns of every block of the pass (block b at
  // V + b * vwords), transposed once before the loop
  uint32_t vall;
  // 1: the pair cohort [0, pair_end) is counted over every block before the
  // loop (tensor GEMM) and its promotions and prunes are precomputed per
  // stop: at stop g <= stop_max the records ev_list[ev_off[g] ..
  // ev_off[g+1]) are promoted, ev_pruned[g] pairs are dropped by the bound,
  // and at stop_max ev_pruned[0] pair boxes complete their pass. Their
  // supports hold the full-pass totals from the start.
  uint32_t pair_events;
  // 1: event-driven loop: every cohort born in the loop is counted over its
  // whole pass at once (k_cohort_pass) and its promotions, erasures and
  // solidifications are tallied per stop in advance: eh_box[s], eh_pruned[s],
  // eh_solid[s] for stops s < ehcap, the first EV_LIST records promoted at s
  // in eb_list[s * EV_LIST ..]. Boxes promoted at a later stop are already in
  // the box set with that stop in cpromo; MAKECANDIDATES treats them as
  // absent until then.
  uint32_t events;
  const uint32_t *ev_off;     // [stop_max + 2]
  const uint32_t *ev_list;    // [pair_end]
  const uint32_t *ev_pruned;  // [stop_max + 1]
  uint32_t *eh_box;           // [ehcap]
  uint32_t *eh_pruned;        // [ehcap]
  uint32_t *eh_solid;         // [ehcap]
  uint32_t *eb_list;          // [ehcap][EV_LIST]
  unsigned long long *ev_work;  // [ehcap] Ctrl.work after the cohort pass of
                                // iteration i (event-driven loop)
  uint32_t ehcap;
  // cohorts of at most cp_records records split each record's blocks over
  // several CTAs: per-block counts in cp_cnt[record][stop_max], the parts
  // done in cp_tick[record] (zero between passes)
  uint32_t cp_records;
  uint32_t *cp_cnt;
  uint32_t *cp_tick;
};

// Records promoted at one stop listed directly by the event-driven loop
// (more are found by a scan of the window).
constexpr uint32_t EV_LIST = 128;
// Largest block count (stop_max) the event-driven loop takes: the cohort
// pass keeps one counter per block in shared memory.
constexpr uint32_t EV_STOPMAX = 8192;

// The column buffer of stop g's block.
__device__ __forceinline__ uint32_t *vcols(const Lattice &L, uint32_t g) {
  if (L.vall) return L.V + (uint64_t)((g - 1) % L.stop_max) * L.vwords;
  return L.V + ((L.vdouble && (g & 1u)) ? L.vwords : 0ull);
}

// First record of the window [head, tail) that the count kernels of stop g
// count themselves: the pair cohort is skipped while the tensor path handles
// it (per-stop GEMM beside the BITSLICE count, or precomputed events).
__device__ __forceinline__ uint32_t counted_lo(const Lattice &L, uint32_t head, uint32_t tail,
                                               uint32_t g, bool bitslice) {
  const uint32_t skip =
      (L.pair_end && g <= L.stop_max && (bitslice || L.pair_events)) ? L.pair_end : 0u;
  return skip > head ? (skip < tail ? skip : tail) : head;
}

// Programmatic dependent launch: every kernel of the stop loop waits for the
// grid before it in the stream (no-op when launched without the attribute)
// and lets the next grid start launching at once.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The pair-cohort kernels of the TENSOR path (GEMM and its PRUNE, which run
// beside the BITSLICE count of the same stop) make the same checks as that
// count, which may stall on the kernel width or the box-set room before
// changing anything; they do nothing when it will stall, so a stop re-run
// after a stall never counts its pairs twice. Reads only values no kernel of
// the stop changes.
__device__ __forceinline__ bool gram_may_run(const Lattice &L, const Ctrl *C, uint32_t kre) {
  if (C->stall || C->done) return false;
  if (C->max_k > kre) return false;
  if ((uint64_t)(C->hash_used + C->n_live) * 2 > L.hcap) return false;
  return C->step <= L.stop_max && C->head == 0;  // the pair cohort is in DASHED
}

// Record index of pair {a, b} (ranks a < b < l1): the first-pass pair join
// writes all pairs of frequent ranks as records 0 .. l1(l1-1)/2 - 1 in
// lexicographic order, before any other record.
__host__ __device__ __forceinline__ uint64_t pair_record(uint64_t a, uint64_t b, uint64_t l1) {
  return a * (2 * l1 - a - 1) / 2 + (b - a - 1);
}

// Block [first, last) of global stop g (1-based), with rewind (Algorithm 2).
__host__ __device__ inline void block_of(uint32_t g, uint32_t stop_max, uint64_t M, uint64_t n,
                                         uint32_t *stop, uint64_t *first, uint64_t *last) {
  uint32_t s = (g - 1) % stop_max + 1;
  *stop = s;
  *first = (uint64_t)(s - 1) * M;
  uint64_t l = (uint64_t)s * M;
  *last = l < n ? l : n;
}

// Set the thread-local text returned by dic_last_error().
void set_last_error(const char *msg);

// Whether the stop-loop launchers give their kernels the programmatic
// dependent launch attribute (a per-host-thread setting: the single-query
// loop turns it on while it enqueues stops that run on one stream, where
// every kernel waits for the one before it with pdl_wait()).
bool &pdl_enabled();

// Launch through cudaLaunchKernelEx with the stop loop's attributes; returns
// this launch's own status.
template <class... KArgs, class... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  if (pdl_enabled()) {
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
}

// ---- kernel launchers (kernels_*.cu) ----
cudaError_t launch_item_count(const uint64_t *B, uint64_t n, uint32_t W, uint32_t m,
                              uint32_t *cnt, cudaStream_t s);
cudaError_t launch_compact_rows(const uint64_t *B, uint64_t n, uint32_t W, const int32_t *rank_of,
                                uint64_t *Bc, uint32_t wc, cudaStream_t s);
cudaError_t launch_pack_csr(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                            uint32_t W, uint64_t *words, uint32_t *bad, cudaStream_t s);
cudaError_t launch_check_padding(const uint64_t *words, uint64_t n, uint32_t m, uint32_t W,
                                 uint32_t *bad, cudaStream_t s);
cudaError_t launch_pair_join(Lattice L, uint64_t npairs, cudaStream_t s);
// Classic DIC (Algorithm 1): every rank as a 1-itemset circle, records 0..l1-1.
cudaError_t launch_singleton_join(Lattice L, cudaStream_t s);
cudaError_t launch_count_rows(Lattice L, int nw, int grid, cudaStream_t s);
cudaError_t launch_promote(Lattice L, int grid, cudaStream_t s);
cudaError_t launch_hash_insert(Lattice L, int grid, cudaStream_t s);
// MAKECANDIDATES followed (in the last block to finish) by the end-of-stop
// bookkeeping: trace row, cohort, CHECKFULLPASS, loop test.
// With slice_next, the same launch also builds the BITSLICE columns of the
// next stop's block (the count of this stop has finished reading them).
// (Lattice.events: MAKECANDIDATES only; the cohort pass closes the stop.)
cudaError_t launch_generate_finish(Lattice L, int grid, bool slice_next, cudaStream_t s);
// Event-driven loop: count the cohort MAKECANDIDATES emitted at the prepared
// stop over its whole pass and tally its events, then close that stop and
// every following one without promotions (at most `budget`) and prepare the
// next stop with promotions (kernels_events.cu). Inside the loop graph
// (`use_cond` 1) it ends the graph's WHILE loop (handle `cond`) when nothing
// is prepared or the iteration limit is reached.
cudaError_t launch_cohort_pass(Lattice L, int grid, uint32_t budget, uint32_t use_cond,
                               unsigned long long cond, cudaStream_t s);
// Hand the loop from the per-stop form to the event-driven one at a stop
// boundary: every live record of three or more items in [lo, tail) is
// counted over the blocks left of its pass, from its count so far, and its
// events are tallied as the cohort pass does (kernels_events.cu). One launch
// takes the records of [lo, hi), at most window_pass_batch(stop_max, n) of
// them, with scratch rows[batch][stop_max] (uninitialised) and tick[batch]
// (zero; left zero).
uint32_t window_pass_batch(uint32_t stop_max, uint32_t nrec);
cudaError_t launch_window_pass(Lattice L, uint32_t lo, uint32_t hi, uint32_t step,
                               uint32_t *rows, uint32_t *tick, int grid, cudaStream_t s);
// Set Ctrl.ev_limit (stream-ordered).
cudaError_t launch_set_ev_limit(Ctrl *C, uint32_t limit, cudaStream_t s);
size_t cohort_pass_smem(uint32_t stop_max, uint32_t l1);
cudaError_t launch_rehash(Lattice L, const uint32_t *oslot, uint32_t ocap, cudaStream_t s);
// The boxes among records [0, tail) in record order: out_idx[0 .. total),
// total = chunk_cnt[collect_chunks(tail)] (chunk_cnt holds
// collect_chunks(tail) + 1 words).
cudaError_t launch_collect_boxes(Lattice L, uint32_t tail, uint32_t *chunk_cnt, uint32_t *out_idx,
                                 cudaStream_t s);
uint32_t collect_chunks(uint32_t tail);
// Size, support and item ids (item_of[rank], at most KRMAX per box, row
// stride KRMAX) of boxes idx[0 .. cnt); masks (row stride wc) when not NULL.
cudaError_t launch_gather_boxes(Lattice L, const uint32_t *idx, uint32_t cnt,
                                const uint32_t *item_of, uint32_t *out_k, uint32_t *out_supp,
                                uint32_t *items, uint64_t *masks, cudaStream_t s);

// Columns of every block of the pass (L.vall), transposed once from the
// original rows B[n][W] (item p -> rank rank_of[p], -1 = not frequent);
// chunk_lo[c] = the number of frequent items below item 512 c, for c = 0 ..
// ceil(W / 8).
cudaError_t launch_slice_all(Lattice L, const uint64_t *B, uint32_t W, const int32_t *rank_of,
                             const uint32_t *chunk_lo, cudaStream_t s);
// All-blocks pair GEMM (L.vall, pairs_lex): pc[b][record] = the pair's count
// over block b (uint32 when `wide`, else uint16: blocks below 65,536 rows).
cudaError_t launch_gram_all_blocks(Lattice L, void *pc, bool wide, cudaStream_t s);
// Pair events from those counts (Lattice pair_events): ev[npairs], hist
// [2 (stop_max + 2)], ev_off [stop_max + 2], cursor [stop_max + 2],
// ev_list [npairs], ev_pruned [stop_max + 1]; writes the pairs' totals.
cudaError_t launch_pair_events(Lattice L, const void *pc, bool wide, uint32_t *ev,
                               uint32_t *hist, uint32_t *ev_off, uint32_t *cursor,
                               uint32_t *ev_list, uint32_t *ev_pruned, cudaStream_t s);

// BITSLICE path (kernels_count_bitslice.cu). V holds the stop's block as
// per-rank bit columns, tile-major: tile t covers rows first+32*TW*t ..,
// V[(t*l1p + r)*stride + w] = rows first+32*(TW*t+w) .. +31 of rank r (bit
// j = row +j); stride = TW+4 (TW = 8, 16) or TW (TW = 4), the extra words
// being padding. l1p = l1 rounded up to a multiple of 4.
size_t bitslice_tile_words(int tw, uint32_t l1p);
// Columns of the block of stop g (g = Ctrl.step when g == 0).
// ahead = 1: the block of the next stop (double-buffered columns only).
cudaError_t launch_slice_block(Lattice L, uint32_t ahead, cudaStream_t s);
// `direct`: the shared-memory-free form for windows expected to be small
// (grid = CTAs of 256 threads); otherwise grid CTAs of 1024 threads.
cudaError_t launch_count_bitslice(Lattice L, const uint32_t *V, int tw, int kre, uint32_t l1p,
                                  uint32_t chunk, uint64_t vwords, int grid, bool direct,
                                  cudaStream_t s);
// CTAs of 256 threads per SM the direct count kernel is built for, by rank
// bucket (its grid is one resident wave).
int count_direct_ctas_per_sm(int kre);
// Windows of at most this many counted records get the direct form.
constexpr uint32_t BS_DIRECT_HOST_MAX = 8192;
// Batched rounds (kernels_batch.cu): one launch per phase for all queries.
cudaError_t launch_batch_plan(const Lattice *Ls, uint32_t Q, bool finish, uint32_t grid,
                              uint32_t chunk_cap, uint32_t *item_prefix, uint32_t *chunk,
                              cudaStream_t s);
cudaError_t launch_batch_count(const Lattice *Ls, uint32_t Q, int tw, int kre,
                               const uint32_t *item_prefix, const uint32_t *chunk,
                               uint32_t smem, int grid, cudaStream_t s);
cudaError_t launch_batch_plan_gen(const Lattice *Ls, uint32_t Q, uint32_t slice_offset,
                                  uint64_t *gen_prefix, uint64_t *slice_prefix, cudaStream_t s);
cudaError_t launch_batch_gen(const Lattice *Ls, uint32_t Q, uint32_t slice_offset,
                             const uint64_t *gen_prefix, const uint64_t *slice_prefix, int grid,
                             cudaStream_t s);

// TENSOR path for the pair cohort (kernels_count_tensor.cu).
uint32_t gram_tile_pairs(uint32_t l1);  // CTAs per K split
uint32_t gram_chunks(uint64_t rows);
// Reads the stop's bit columns L.V (so it needs L.tw in {4, 8, 16}); does
// nothing when the BITSLICE count of the same stop (kre ranks) will stall,
// so a re-run stop never counts its pairs twice.
cudaError_t launch_gram_pairs(Lattice L, uint32_t nsplit, uint32_t kre, cudaStream_t s);

// PRUNE for the pair cohort counted by the tensor path (one thread per record).
cudaError_t launch_settle_pairs(Lattice L, int grid, uint32_t kre, cudaStream_t s);

// Association rules (kernels_rules.cu): insert the itemsets into a table,
// then evaluate every split of every itemset of >= 2 items; rules go to
// out_* at an atomic cursor; err bit 0 = an itemset's subset is missing,
// bit 1 = table full.
cudaError_t launch_rules(const uint64_t *masks, const uint32_t *k, const uint32_t *supp,
                         const uint64_t *work_prefix, uint32_t *hslot, uint64_t count,
                         uint32_t W, uint32_t hcap, uint32_t num, uint32_t den, uint64_t total,
                         unsigned long long *cursor, uint32_t *out_z, uint32_t *out_code,
                         uint32_t *out_sx, uint32_t *err, cudaStream_t s);

// Largest candidate chunk whose bitslice shared-memory footprint fits.
uint32_t bitslice_max_chunk(int tw, int kre, uint32_t l1p, size_t smem_limit);
size_t bitslice_smem(int tw, int kre, uint32_t l1p, uint32_t chunk);

// Width bucket (max nonzero 32-bit halves per candidate) the rows kernel
// needs for itemsets of up to max_k items in wc-word masks.
int rows_width_bucket(uint32_t max_k, uint32_t wc);

}  // namespace dic
