// COUNTSUPPORT (Algorithm 3), BITSLICE path.
//
// The containment test of Section 4.1 asks, for every candidate C and row T
// of the block, whether every item of C is set in T. Transposing the block
// into one bit column per frequent item (32 rows per word) turns the test of
// 32 rows at once into an AND of C's k column words, and the count of
// contained rows into popc of that AND. The set of (candidate, row) tests and
// every support are exactly those of the row-wise test; only the order in
// which the bits are combined changes.
//
// Per stop:
//   k_slice_block    rows [first, last) of the compacted bitmaps -> V, the
//                    columns of every rank, tile-major and padded so that a
//                    tile is one contiguous, shared-memory-ready byte range.
//   k_count_bitslice each CTA owns a contiguous chunk of the candidate
//                    window; it streams the V tiles through a double buffer
//                    (cp.async) and every thread ANDs and popcounts its
//                    candidates' columns with 128-bit shared loads. Counts
//                    stay in shared memory until the chunk is done; then each
//                    record's support is written once and PRUNE (Algorithm
//                    4) is applied to it in the same pass, inserting new
//                    boxes into the box set. Windows of at most
//                    BS_DIRECT_MAX records are counted a warp per record
//                    straight from the (L2-resident) columns instead.
//   k_count_direct   that direct form alone, without shared memory, for
//                    windows the host expects to be small.
//   k_settle_pairs   PRUNE of the pair cohort the tensor path counted.
//
// Tile rows are padded to 16-byte multiples (TW+4 words for TW = 8, 16; TW
// for TW = 4) so that eight threads reading consecutive ranks with 128-bit
// loads hit distinct banks.
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"
#include "lattice_device.cuh"
#include "bitslice_device.cuh"

namespace dic {

constexpr int BS_THREADS = 1024;

// ------------------------------------------------------------ transpose
// Standalone form: the first stop of a run or a resumed stop, and, with
// double-buffered columns, the next stop's block while this one is counted
// (otherwise the previous stop's generate kernel transposes it).
__global__ void __launch_bounds__(256) k_slice_block(Lattice L, uint32_t ahead) {
  pdl_wait();
  pdl_trigger();
  Ctrl *C = L.ctrl;
  if (C->stall || C->done) return;
  slice_block_warps(L, C->step + ahead,
                    (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                    (uint64_t)gridDim.x * (blockDim.x >> 5));
}

cudaError_t launch_slice_block(Lattice L, uint32_t ahead, cudaStream_t s) {
  const uint64_t blockmax = L.M < L.n ? L.M : L.n;
  const uint64_t nw32 = (blockmax + 31) / 32;
  const uint64_t items = ((nw32 + L.tw - 1) / L.tw) * L.tw * L.wc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t want = (items + 7) / 8;
  int grid = (int)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
  if (grid < 1) grid = 1;
  return launch_k(k_slice_block, grid, 256, 0, s, L, ahead);
}

// Every block of the pass at once (L.vall). A CTA takes one (block b, tile t,
// chunk of SJC source words) item: it stages the tile's TW*32 rows x SJC
// words of the original rows B[n][W] in shared memory (row-contiguous,
// coalesced loads; rows past the block's end read as 0), transposes each
// 32-row word across a warp (bit i of source word j is item 64j + i), keeps
// the columns of the frequent items at their ranks in a shared output tile,
// and writes that tile's rank rows (TW words each) out contiguously. The
// chunk's frequent items have the consecutive ranks chunk_lo[c] ..
// chunk_lo[c+1] - 1 (rank order is item order). An index outside V is
// recorded in Ctrl.error and skipped.
constexpr uint32_t SJC = 8;                      // source words per chunk
constexpr uint32_t SROWPAD = SJC + 1;            // padded staged row (words)
constexpr uint32_t SRANKS = SJC * 64;            // items (at most ranks) per chunk

size_t slice_all_smem(uint32_t tw) {
  return (size_t)tw * 32 * SROWPAD * 8 + (size_t)SRANKS * (tw + 1) * 4 + SRANKS * 4;
}

constexpr uint32_t SLICE_THREADS = 256;

template <uint32_t TW>
__global__ void __launch_bounds__(SLICE_THREADS) k_slice_all(Lattice L, const uint64_t *__restrict__ B,
                                                   uint32_t W,
                                                   const int32_t *__restrict__ rank_of,
                                                   const uint32_t *__restrict__ chunk_lo) {
  extern __shared__ __align__(16) uint8_t ssm[];
  constexpr uint32_t ST = bs_stride((int)TW), ROWS = TW * 32, OS = TW + 1;
  const uint32_t l1p = L.l1p;
  uint64_t *sin = reinterpret_cast<uint64_t *>(ssm);                   // [ROWS][SROWPAD]
  uint32_t *sout = reinterpret_cast<uint32_t *>(sin + (size_t)ROWS * SROWPAD);  // [SRANKS][OS]
  int32_t *srank = reinterpret_cast<int32_t *>(sout + (size_t)SRANKS * OS);  // [SRANKS]
  const uint64_t blockmax = L.M < L.n ? L.M : L.n;
  const uint32_t ntiles = (uint32_t)(((blockmax + 31) / 32 + TW - 1) / TW);
  const uint32_t nch = (W + SJC - 1) / SJC;
  const uint64_t items = (uint64_t)L.stop_max * ntiles * nch;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const uint64_t b = it / ((uint64_t)ntiles * nch);
    const uint32_t rem = (uint32_t)(it % ((uint64_t)ntiles * nch));
    const uint32_t t = rem / nch, c = rem % nch;
    const uint32_t j0 = c * SJC;
    const uint64_t first = b * L.M;
    const uint64_t last = first + L.M < L.n ? first + L.M : L.n;
    const uint64_t row0 = first + (uint64_t)t * ROWS;
    const uint32_t rlo = chunk_lo[c], rhi = chunk_lo[c + 1];
    __syncthreads();  // the previous item's tiles are free
    {
      // every load of the tile issued before any is stored (the launch has
      // SLICE_THREADS threads)
      constexpr uint32_t NL = ROWS * SJC / SLICE_THREADS;
      uint64_t v[NL];
#pragma unroll
      for (uint32_t i = 0; i < NL; ++i) {
        const uint32_t e = threadIdx.x + i * SLICE_THREADS;
        const uint32_t r = e / SJC, w = e % SJC;
        const uint64_t row = row0 + r;
        v[i] = (row < last && j0 + w < W) ? __ldcs(B + row * W + j0 + w) : 0ull;
      }
#pragma unroll
      for (uint32_t i = 0; i < NL; ++i) {
        const uint32_t e = threadIdx.x + i * SLICE_THREADS;
        sin[(e / SJC) * SROWPAD + e % SJC] = v[i];
      }
    }
    for (uint32_t e = threadIdx.x; e < SRANKS; e += blockDim.x)
      srank[e] = j0 * 64 + e < W * 64 ? __ldg(rank_of + j0 * 64 + e) : -1;
    __syncthreads();
#pragma unroll 4
    for (uint32_t q = warp; q < TW * SJC; q += nwarp) {
      const uint32_t g = q / SJC, j = q % SJC;
      const uint64_t x = sin[(g * 32 + lane) * SROWPAD + j];
      const uint32_t lo = warp_transpose32((uint32_t)x);
      const uint32_t hi = warp_transpose32((uint32_t)(x >> 32));
      const int32_t r0 = srank[j * 64 + lane], r1 = srank[j * 64 + 32 + lane];
      if (r0 >= 0) sout[((uint32_t)r0 - rlo) * OS + g] = lo;
      if (r1 >= 0) sout[((uint32_t)r1 - rlo) * OS + g] = hi;
    }
    __syncthreads();
    // each rank's ST words of this tile (its TW words, then the padding as
    // zeros), four per 16-byte store: a tile row starts on a 16-byte
    // boundary (ST words are a multiple of four), and writing the padding
    // too leaves no 32-byte sector partly written (a partial sector costs
    // the memory a read before the write)
    uint32_t *Vb = L.V + b * L.vwords;
    constexpr uint32_t SQ = ST / 4;
    const uint32_t nq = (rhi - rlo) * SQ;
    for (uint32_t e = threadIdx.x; e < nq; e += blockDim.x) {
      const uint32_t rr = e / SQ, w = 4 * (e % SQ);
      const uint64_t idx = ((uint64_t)t * l1p + rlo + rr) * ST + w;
      if (idx + 3 < L.vwords && rlo + rr < l1p && rr < SRANKS) {
        const uint32_t *src = sout + rr * OS + w;
        *reinterpret_cast<uint4 *>(Vb + idx) =
            w < TW ? make_uint4(src[0], src[1], src[2], src[3]) : make_uint4(0u, 0u, 0u, 0u);
      } else {
        L.ctrl->error = DIC_INTERNAL_BOUNDS;
      }
    }
  }
}

cudaError_t launch_slice_all(Lattice L, const uint64_t *B, uint32_t W, const int32_t *rank_of,
                             const uint32_t *chunk_lo, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = slice_all_smem(L.tw);
  void (*kern)(Lattice, const uint64_t *, uint32_t, const int32_t *, const uint32_t *) =
      L.tw == 16 ? k_slice_all<16> : L.tw == 8 ? k_slice_all<8> : k_slice_all<4>;
  if (L.tw != 16 && L.tw != 8 && L.tw != 4) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<sms * 3, SLICE_THREADS, smem, s>>>(L, B, W, rank_of, chunk_lo);
  return cudaGetLastError();
}

size_t bitslice_tile_words(int tw, uint32_t l1p) { return (size_t)l1p * bs_stride(tw); }

size_t bitslice_smem(int tw, int kre, uint32_t l1p, uint32_t chunk) {
  const size_t tile = bitslice_tile_words(tw, l1p) * 4;
  return 2 * tile + (size_t)chunk * (2 * kre + 4 + 1) + 16;
}

uint32_t bitslice_max_chunk(int tw, int kre, uint32_t l1p, size_t smem_limit) {
  // the count kernels' static shared memory (block tallies) comes out of the
  // same per-block limit
  constexpr size_t kStaticReserve = 1024;
  smem_limit = smem_limit > kStaticReserve ? smem_limit - kStaticReserve : 0;
  const size_t tile = bitslice_tile_words(tw, l1p) * 4;
  if (2 * tile + 16 >= smem_limit) return 0;
  size_t c = (smem_limit - 2 * tile - 16) / (2 * kre + 4 + 1);
  c &= ~(size_t)3;
  return c > 0x7fffffff ? 0x7fffffff : (uint32_t)c;
}

template <int TW, int KRE>
__global__ void __launch_bounds__(BS_THREADS) k_count_bitslice(Lattice L,
                                                               const uint32_t *__restrict__ V,
                                                               uint32_t l1p, uint32_t chunk_cap,
                                                               uint64_t vwords) {
  extern __shared__ __align__(16) uint32_t sm[];
  pdl_wait();
  pdl_trigger();
  Ctrl *C = L.ctrl;
  uint32_t ev[3];
  const StopState cs = cta_stop_state(L, C, ev);
  if (cs.stall || cs.done) return;
  if (!bs_checks_v<KRE>(L, C, cs.max_k, cs.hash_used, cs.n_live, blockIdx.x == 0)) return;
  const uint32_t g = cs.step;
  uint32_t nw32, ntiles;
  if (!bs_block_tiles<TW>(L, C, g, &nw32, &ntiles)) return;
  const uint32_t head = cs.head, tail = cs.tail;
  // records below the pair cohort's end, while the tensor path has it, are
  // counted and pruned there; this kernel counts [lo, tail)
  const uint32_t lo = counted_lo(L, head, tail, g, true);
  const uint32_t ncand = tail - lo;
  uint32_t pruned = 0, solid = 0;
  unsigned long long work = 0;
  apply_pair_events_range(L, C, g, ev, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                          (uint64_t)gridDim.x * blockDim.x, pruned, solid);
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) stage_next_events(L, C, g);
  if (ncand == 0) {
    block_add_tallies(C, pruned, solid, work);
    return;
  }
  if (ncand <= BS_DIRECT_MAX) {
    // few candidates: no shared tiles; a warp per candidate ANDs its columns
    // straight from the (L2-resident) column buffer
    bs_count_direct<TW, KRE>(L, C, g, lo, tail, nw32, pruned, solid, work);
  } else {
    uint32_t chunk = (ncand + gridDim.x - 1) / gridDim.x;
    chunk = (chunk + 3) & ~3u;
    if (chunk < 4) chunk = 4;
    if (chunk > chunk_cap) chunk = chunk_cap;
    const uint32_t nchunks = (ncand + chunk - 1) / chunk;
    for (uint32_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
      const uint32_t c0 = lo + ch * chunk;
      const uint32_t cn = (tail - c0) < chunk ? (tail - c0) : chunk;
      bs_count_chunk<TW, KRE, BS_THREADS>(L, C, g, c0, cn, nw32, ntiles, sm, chunk_cap, pruned,
                                          solid, work);
    }
  }
  block_add_tallies(C, pruned, solid, work);
  (void)V; (void)l1p; (void)vwords;
}

// The same count for a window the host expects to be small: direct mode
// only (it is exact at any window size), no shared memory, so its CTAs can
// share SMs with the pair-cohort GEMM of the same stop.
// Three CTAs per SM for itemsets of at most four items (three 16-byte
// loads per rank in flight: 96 x 4 words cover a 12,288-row block in one
// round, at most 85 registers); one for longer ones, whose unrolled rank
// loads take more registers than two CTAs per SM leave.
__host__ __device__ constexpr int direct_ctas_per_sm(int kre) { return kre <= 4 ? 3 : 1; }
__host__ __device__ constexpr uint32_t direct_unroll(int kre) { return kre <= 4 ? 3u : 4u; }
int count_direct_ctas_per_sm(int kre) { return direct_ctas_per_sm(kre); }

template <int TW, int KRE>
__global__ void __launch_bounds__(256, direct_ctas_per_sm(KRE)) k_count_direct(Lattice L) {
  pdl_wait();
  pdl_trigger();
  Ctrl *C = L.ctrl;
  uint32_t ev[3];
  const StopState cs = cta_stop_state(L, C, ev);
  if (cs.stall || cs.done) return;
  if (!bs_checks_v<KRE>(L, C, cs.max_k, cs.hash_used, cs.n_live, blockIdx.x == 0)) return;
  const uint32_t g = cs.step;
  uint32_t nw32, ntiles;
  if (!bs_block_tiles<TW>(L, C, g, &nw32, &ntiles)) return;
  const uint32_t head = cs.head, tail = cs.tail;
  const uint32_t lo = counted_lo(L, head, tail, g, true);
  uint32_t pruned = 0, solid = 0;
  unsigned long long work = 0;
  apply_pair_events_range(L, C, g, ev, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                          (uint64_t)gridDim.x * blockDim.x, pruned, solid);
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) stage_next_events(L, C, g);
  if (lo < tail)
    bs_count_direct<TW, KRE, direct_unroll(KRE)>(L, C, g, lo, tail, nw32, pruned, solid, work);
  block_add_tallies(C, pruned, solid, work);
}

// PRUNE (Algorithm 4) for the pair cohort after the tensor kernel has added
// this stop's counts: four records per thread, every load issued before any
// record is examined.
__global__ void __launch_bounds__(256) k_settle_pairs(Lattice L, uint32_t kre) {
  pdl_wait();
  pdl_trigger();
  Ctrl *C = L.ctrl;
  if (!L.pair_end || !gram_may_run(L, C, kre)) return;
  const uint32_t g = C->step;
  const uint32_t head = C->head, end = L.pair_end < C->tail ? L.pair_end : C->tail;
  uint32_t pruned = 0, solid = 0;
  // four records per thread, all loads issued before any is used
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t c = head + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < end;
       c += 4 * stride) {
    uint8_t sh[4];
    uint32_t sp[4], bi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint64_t cc = c + u * stride;
      const bool in = cc < end;
      sh[u] = in ? L.cshape[cc] : (uint8_t)SH_NIL;
      sp[u] = in ? L.csupp[cc] : 0u;
      bi[u] = in ? L.cbirth[cc] : 0u;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      settle_loaded(L, C, (uint32_t)(c + u * stride), sh[u], bi[u], sp[u], g, true, pruned,
                    solid);
  }
  block_add_tallies(C, pruned, solid, 0ull);
}

cudaError_t launch_settle_pairs(Lattice L, int grid, uint32_t kre, cudaStream_t s) {
  return launch_k(k_settle_pairs, grid, 256, 0, s, L, kre);
}

template <int TW, int KRE>
static cudaError_t go(Lattice L, const uint32_t *V, uint32_t l1p, uint32_t chunk, uint64_t vw,
                      int grid, bool direct, cudaStream_t s) {
  if (direct) return launch_k(k_count_direct<TW, KRE>, grid, 256, 0, s, L);
  const size_t smem = bitslice_smem(TW, KRE, l1p, chunk);
  cudaError_t e = cudaFuncSetAttribute(k_count_bitslice<TW, KRE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_k(k_count_bitslice<TW, KRE>, grid, BS_THREADS, smem, s, L, V, l1p, chunk, vw);
}

template <int TW>
static cudaError_t go_k(Lattice L, const uint32_t *V, int kre, uint32_t l1p, uint32_t chunk,
                        uint64_t vw, int grid, bool direct, cudaStream_t s) {
  switch (kre) {
    case 2: return go<TW, 2>(L, V, l1p, chunk, vw, grid, direct, s);
    case 4: return go<TW, 4>(L, V, l1p, chunk, vw, grid, direct, s);
    case 8: return go<TW, 8>(L, V, l1p, chunk, vw, grid, direct, s);
    default: return go<TW, 16>(L, V, l1p, chunk, vw, grid, direct, s);
  }
}

cudaError_t launch_count_bitslice(Lattice L, const uint32_t *V, int tw, int kre, uint32_t l1p,
                                  uint32_t chunk, uint64_t vwords, int grid, bool direct,
                                  cudaStream_t s) {
  if (tw != 16 && tw != 8 && tw != 4) return cudaErrorInvalidValue;
  if (bitslice_tile_words(tw, l1p) % 4) return cudaErrorInvalidValue;
  switch (tw) {
    case 16: return go_k<16>(L, V, kre, l1p, chunk, vwords, grid, direct, s);
    case 8: return go_k<8>(L, V, kre, l1p, chunk, vwords, grid, direct, s);
    default: return go_k<4>(L, V, kre, l1p, chunk, vwords, grid, direct, s);
  }
}

}  // namespace dic
