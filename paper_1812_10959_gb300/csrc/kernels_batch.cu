// Batched stops: many independent queries (database, minsup, M), each with
// its own lattice, advance one stop of Algorithm 2 per round, and every phase
// of a round is ONE launch over all queries:
//
//   k_batch_count    persistent BITSLICE count over (query, candidate chunk)
//                    work items, PRUNE applied in the epilogue
//   k_batch_plan_gen per-query generation / next-block transpose work
//   k_batch_gen      MAKECANDIDATES for every query + the next stop's bit
//                    columns of every query
//   k_batch_plan     closes the stop of every query that ran one
//                    (CHECKFULLPASS, trace, loop test) and lays out the next
//                    round's count work items
//
// A query whose stop stalls (a buffer to grow) or whose itemsets outgrow the
// BITSLICE ranks drops out of the batched kernels (they skip it) until the
// host has recovered it; a query marked `solo` is never touched by them.
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"
#include "lattice_device.cuh"
#include "bitslice_device.cuh"

namespace dic {

constexpr int PLAN_THREADS = 1024;
constexpr int BATCH_COUNT_THREADS = 1024;

__device__ __forceinline__ bool batch_active(const Ctrl *C) {
  return !C->done && !C->stall && !C->solo && !C->error;
}

// Largest q with prefix[q] <= x (prefix non-decreasing, prefix[0] = 0).
template <class T>
__device__ __forceinline__ uint32_t find_query(const T *prefix, uint32_t Q, T x) {
  uint32_t lo = 0, hi = Q;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (prefix[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Block-wide exclusive scan of one value per thread slot over Q queries (Q
// may exceed the block: each thread owns a contiguous run of queries).
template <class T>
__device__ void block_prefix(T *prefix, uint32_t Q, T (*value)(const Lattice &, uint32_t, uint32_t,
                                                                 uint32_t),
                             const Lattice *Ls, uint32_t a, uint32_t b) {
  __shared__ T part[PLAN_THREADS];
  const uint32_t per = (Q + PLAN_THREADS - 1) / PLAN_THREADS;
  const uint32_t q0 = threadIdx.x * per, q1 = q0 + per < Q ? q0 + per : Q;
  T sum = 0;
  for (uint32_t q = q0; q < q1; ++q) sum += value(Ls[q], q, a, b);
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    T run = 0;
    for (int i = 0; i < PLAN_THREADS; ++i) {
      const T v = part[i];
      part[i] = run;
      run += v;
    }
    prefix[Q] = run;
  }
  __syncthreads();
  T run = part[threadIdx.x];
  for (uint32_t q = q0; q < q1; ++q) {
    prefix[q] = run;
    run += value(Ls[q], q, a, b);
  }
  __syncthreads();
}

__device__ uint32_t count_items(const Lattice &L, uint32_t, uint32_t chunk, uint32_t) {
  const Ctrl *C = L.ctrl;
  if (!batch_active(C)) return 0;
  const uint32_t win = C->tail - C->head;
  return (win + chunk - 1) / chunk;
}

__device__ uint64_t gen_items(const Lattice &L, uint32_t, uint32_t, uint32_t) {
  const Ctrl *C = L.ctrl;
  if (!batch_active(C)) return 0;
  return (uint64_t)C->n_newbox * L.l1;
}

__device__ uint64_t slice_items(const Lattice &L, uint32_t, uint32_t offset, uint32_t) {
  const Ctrl *C = L.ctrl;
  if (!batch_active(C) || !L.V) return 0;
  uint32_t stop;
  uint64_t first, last;
  block_of(C->step + offset, L.stop_max, L.M, L.n, &stop, &first, &last);
  const uint64_t nw32 = (last - first + 31) / 32;
  return ((nw32 + L.tw - 1) / L.tw) * L.tw * L.wc;
}

// Close the stop every active query just ran (finish != 0), then lay out the
// next count: one chunk size for all queries (the total window spread over
// about two items per CTA) and the per-query prefix of items.
__global__ void __launch_bounds__(PLAN_THREADS) k_batch_plan(const Lattice *Ls, uint32_t Q,
                                                             int finish, uint32_t grid,
                                                             uint32_t chunk_cap,
                                                             uint32_t *item_prefix,
                                                             uint32_t *chunk_out) {
  __shared__ unsigned long long total;
  if (threadIdx.x == 0) total = 0;
  __syncthreads();
  unsigned long long mine = 0;
  for (uint32_t q = threadIdx.x; q < Q; q += PLAN_THREADS) {
    Ctrl *C = Ls[q].ctrl;
    if (finish && batch_active(C)) finish_stop(Ls[q], C);
    if (batch_active(C)) mine += C->tail - C->head;
  }
  atomicAdd(&total, mine);
  __syncthreads();
  uint64_t chunk = (total + 2ull * grid - 1) / (2ull * grid);
  chunk = (chunk + 3) & ~3ull;
  if (chunk < 64) chunk = 64;
  if (chunk > chunk_cap) chunk = chunk_cap;
  if (threadIdx.x == 0) *chunk_out = (uint32_t)chunk;
  block_prefix<uint32_t>(item_prefix, Q, count_items, Ls, (uint32_t)chunk, 0);
}

template <int TW, int KRE>
__global__ void __launch_bounds__(BATCH_COUNT_THREADS) k_batch_count(
    const Lattice *Ls, uint32_t Q, const uint32_t *item_prefix, const uint32_t *chunk_in,
    uint32_t smem_bytes) {
  extern __shared__ __align__(16) uint32_t sm[];
  const uint32_t total = item_prefix[Q];
  const uint32_t chunk = *chunk_in;
  for (uint32_t item = blockIdx.x; item < total; item += gridDim.x) {
    const uint32_t q = find_query<uint32_t>(item_prefix, Q, item);
    const Lattice L = Ls[q];
    Ctrl *C = L.ctrl;
    const uint32_t ch = item - item_prefix[q];
    if (!bs_checks<KRE>(L, C, ch == 0)) continue;
    const uint32_t g = C->step;
    uint32_t nw32, ntiles;
    if (!bs_block_tiles<TW>(L, C, g, &nw32, &ntiles)) continue;
    // this query's chunk capacity in the launch's shared memory
    const uint32_t tile_bytes = L.l1p * bs_stride(TW) * 4;
    const uint32_t cap = (smem_bytes - 2 * tile_bytes - 16) / (2 * KRE + 5) & ~3u;
    const uint32_t c0 = C->head + ch * chunk;
    const uint32_t cn = (C->tail - c0) < chunk ? (C->tail - c0) : chunk;
    if (cn > cap) {  // internal sizing error: record, skip
      if (threadIdx.x == 0) C->error = DIC_INTERNAL_BOUNDS;
      continue;
    }
    uint32_t pruned = 0, solid = 0;
    unsigned long long work = 0;
    bs_count_chunk<TW, KRE, BATCH_COUNT_THREADS>(L, C, g, c0, cn, nw32, ntiles, sm, cap, pruned,
                                                 solid, work);
    block_add_tallies(C, pruned, solid, work);  // (the item is the CTA's alone)
  }
}

__global__ void __launch_bounds__(PLAN_THREADS) k_batch_plan_gen(const Lattice *Ls, uint32_t Q,
                                                                 uint32_t slice_offset,
                                                                 uint64_t *gen_prefix,
                                                                 uint64_t *slice_prefix) {
  block_prefix<uint64_t>(gen_prefix, Q, gen_items, Ls, 0, 0);
  block_prefix<uint64_t>(slice_prefix, Q, slice_items, Ls, slice_offset, 0);
}

// Transposes (warp items) the block of stop step+slice_offset of every
// active query, then runs MAKECANDIDATES (thread items) for every query.
__global__ void __launch_bounds__(256) k_batch_gen(const Lattice *Ls, uint32_t Q,
                                                   uint32_t slice_offset,
                                                   const uint64_t *gen_prefix,
                                                   const uint64_t *slice_prefix) {
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t wid = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint64_t stotal = slice_prefix[Q];
  for (uint64_t it = wid; it < stotal; it += nwarps) {
    const uint32_t q = find_query<uint64_t>(slice_prefix, Q, it);
    const Lattice &L = Ls[q];
    // one (word, mask word) item of this query: slice_block_warps with a
    // single-item range
    slice_block_warps(L, L.ctrl->step + slice_offset, it - slice_prefix[q], ~0ull >> 1);
  }
  const uint64_t gtotal = gen_prefix[Q];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < gtotal; w += stride) {
    const uint32_t q = find_query<uint64_t>(gen_prefix, Q, w);
    const Lattice &L = Ls[q];
    Ctrl *C = L.ctrl;
    const uint64_t local = w - gen_prefix[q];
    gen_candidate(L, C, (uint32_t)(local / L.l1), (uint32_t)(local % L.l1), C->step, C->tail);
  }
}

// ------------------------------------------------------------- launchers
cudaError_t launch_batch_plan(const Lattice *Ls, uint32_t Q, bool finish, uint32_t grid,
                              uint32_t chunk_cap, uint32_t *item_prefix, uint32_t *chunk,
                              cudaStream_t s) {
  k_batch_plan<<<1, PLAN_THREADS, 0, s>>>(Ls, Q, finish ? 1 : 0, grid, chunk_cap, item_prefix,
                                          chunk);
  return cudaGetLastError();
}

template <int TW, int KRE>
static cudaError_t go_batch(const Lattice *Ls, uint32_t Q, const uint32_t *item_prefix,
                            const uint32_t *chunk, uint32_t smem, int grid, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_batch_count<TW, KRE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_batch_count<TW, KRE><<<grid, BATCH_COUNT_THREADS, smem, s>>>(Ls, Q, item_prefix, chunk, smem);
  return cudaGetLastError();
}

cudaError_t launch_batch_count(const Lattice *Ls, uint32_t Q, int tw, int kre,
                               const uint32_t *item_prefix, const uint32_t *chunk,
                               uint32_t smem, int grid, cudaStream_t s) {
#define DIC_BATCH_KRE(TWV)                                                     \
  switch (kre) {                                                               \
    case 2: return go_batch<TWV, 2>(Ls, Q, item_prefix, chunk, smem, grid, s); \
    case 4: return go_batch<TWV, 4>(Ls, Q, item_prefix, chunk, smem, grid, s); \
    case 8: return go_batch<TWV, 8>(Ls, Q, item_prefix, chunk, smem, grid, s); \
    default: return go_batch<TWV, 16>(Ls, Q, item_prefix, chunk, smem, grid, s); \
  }
  switch (tw) {
    case 16: DIC_BATCH_KRE(16)
    case 8: DIC_BATCH_KRE(8)
    default: DIC_BATCH_KRE(4)
  }
#undef DIC_BATCH_KRE
}

cudaError_t launch_batch_plan_gen(const Lattice *Ls, uint32_t Q, uint32_t slice_offset,
                                  uint64_t *gen_prefix, uint64_t *slice_prefix, cudaStream_t s) {
  k_batch_plan_gen<<<1, PLAN_THREADS, 0, s>>>(Ls, Q, slice_offset, gen_prefix, slice_prefix);
  return cudaGetLastError();
}

cudaError_t launch_batch_gen(const Lattice *Ls, uint32_t Q, uint32_t slice_offset,
                             const uint64_t *gen_prefix, const uint64_t *slice_prefix, int grid,
                             cudaStream_t s) {
  k_batch_gen<<<grid, 256, 0, s>>>(Ls, Q, slice_offset, gen_prefix, slice_prefix);
  return cudaGetLastError();
}

}  // namespace dic
