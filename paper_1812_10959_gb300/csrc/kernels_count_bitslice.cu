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
//                    boxes into the box set.
//
// Tile rows are padded to 16-byte multiples (TW+4 words for TW = 8, 16; TW
// for TW = 4) so that eight threads reading consecutive ranks with 128-bit
// loads hit distinct banks.
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"
#include "lattice_device.cuh"

namespace dic {

constexpr int BS_THREADS = 1024;

// ------------------------------------------------------------ transpose
// Standalone form (first stop of a run, or a resumed stop); later stops get
// their columns from the previous stop's generate kernel.
__global__ void __launch_bounds__(256) k_slice_block(Lattice L) {
  Ctrl *C = L.ctrl;
  if (C->stall || C->done) return;
  slice_block_warps(L, C->step, (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5),
                    (uint64_t)gridDim.x * (blockDim.x >> 5));
}

cudaError_t launch_slice_block(Lattice L, cudaStream_t s) {
  const uint64_t blockmax = L.M < L.n ? L.M : L.n;
  const uint64_t nw32 = (blockmax + 31) / 32;
  const uint64_t items = ((nw32 + L.tw - 1) / L.tw) * L.tw * L.wc;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t want = (items + 7) / 8;
  int grid = (int)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
  if (grid < 1) grid = 1;
  k_slice_block<<<grid, 256, 0, s>>>(L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- count
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

size_t bitslice_tile_words(int tw, uint32_t l1p) { return (size_t)l1p * bs_stride(tw); }

size_t bitslice_smem(int tw, int kre, uint32_t l1p, uint32_t chunk) {
  const size_t tile = bitslice_tile_words(tw, l1p) * 4;
  return 2 * tile + (size_t)chunk * (2 * kre + 4 + 1) + 16;
}

uint32_t bitslice_max_chunk(int tw, int kre, uint32_t l1p, size_t smem_limit) {
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
  constexpr uint32_t ST = bs_stride(TW);
  constexpr int NV = TW / 4;  // 128-bit loads per rank and tile
  Ctrl *C = L.ctrl;
  if (C->stall || C->done) return;
  if (C->max_k > (uint32_t)KRE) {
    if (blockIdx.x == 0 && threadIdx.x == 0) C->stall = ST_WIDTH;
    return;
  }
  // room in the box set for every live record, checked before any change
  if ((uint64_t)(C->hash_used + C->n_live) * 2 > L.hcap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) C->stall = ST_HASH_COUNT;
    return;
  }
  const uint32_t tile_words = l1p * ST;
  uint32_t *S0 = sm;
  uint32_t *S1 = sm + tile_words;
  uint16_t *rk = reinterpret_cast<uint16_t *>(sm + 2 * tile_words);
  uint32_t *cnt = reinterpret_cast<uint32_t *>(rk + (size_t)chunk_cap * KRE);
  uint8_t *kk = reinterpret_cast<uint8_t *>(cnt + chunk_cap);

  const uint32_t g = C->step;
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  const uint32_t nw32 = (uint32_t)((last - first + 31) / 32);
  const uint32_t ntiles = (nw32 + TW - 1) / TW;
  if ((uint64_t)ntiles * tile_words > vwords) {  // internal sizing error: record, skip
    if (threadIdx.x == 0) C->error = DIC_INTERNAL_BOUNDS;
    return;
  }
  const uint32_t head = C->head, tail = C->tail;
  const uint32_t ncand = tail - head;
  // balance the live window over the grid; shared memory holds chunk_cap
  uint32_t chunk = (ncand + gridDim.x - 1) / gridDim.x;
  chunk = (chunk + 3) & ~3u;
  if (chunk < 4) chunk = 4;
  if (chunk > chunk_cap) chunk = chunk_cap;
  const uint32_t nchunks = (ncand + chunk - 1) / chunk;
  const uint32_t tid = threadIdx.x;
  uint32_t pruned = 0, solid = 0;

  for (uint32_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const uint32_t c0 = head + ch * chunk;
    const uint32_t cn = (tail - c0) < chunk ? (tail - c0) : chunk;
    __syncthreads();  // shared memory of the previous chunk is free
    for (uint32_t o = tid * 4; o < tile_words; o += BS_THREADS * 4) cp_async16(S0 + o, V + o);
    cp_async_commit();
    for (uint32_t i = tid; i < cn; i += BS_THREADS) {
      const uint32_t c = c0 + i;
      const uint32_t k = L.cshape[c] == SH_NIL ? 0u : (uint32_t)L.ck[c];
      kk[i] = (uint8_t)k;
      cnt[i] = 0;
#pragma unroll
      for (int q = 0; q < KRE; ++q)
        rk[(size_t)i * KRE + q] = (uint32_t)q < k ? L.cranks[(uint64_t)c * KRMAX + q] : (uint16_t)0;
    }
    for (uint32_t t = 0; t < ntiles; ++t) {
      if (t + 1 < ntiles) {
        uint32_t *dst = ((t + 1) & 1) ? S1 : S0;
        const uint32_t *src = V + (size_t)(t + 1) * tile_words;
        for (uint32_t o = tid * 4; o < tile_words; o += BS_THREADS * 4) cp_async16(dst + o, src + o);
      }
      cp_async_commit();
      cp_async_wait_1();
      __syncthreads();
      const uint32_t *S = (t & 1) ? S1 : S0;
      for (uint32_t i = tid; i < cn; i += BS_THREADS) {
        const uint32_t k = kk[i];
        if (k == 0) continue;
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
    unsigned long long work = 0;
    for (uint32_t i = tid; i < cn; i += BS_THREADS) {
      if (!kk[i]) continue;
      const uint32_t c = c0 + i;
      const uint32_t s = L.csupp[c] + cnt[i];
      L.csupp[c] = s;
      settle_record(L, C, c, s, g, true, pruned, solid);
      // algorithmic work: k-1 AND + POPC + ADD per 32-row word
      work += (unsigned long long)(kk[i] + 1) * nw32;
    }
    warp_add_u64(&C->work, work);
  }
  if (pruned) atomicAdd(&C->n_pruned, pruned);
  if (solid) atomicAdd(&C->n_solid, solid);
}

template <int TW, int KRE>
static cudaError_t go(Lattice L, const uint32_t *V, uint32_t l1p, uint32_t chunk, uint64_t vw,
                      int grid, cudaStream_t s) {
  const size_t smem = bitslice_smem(TW, KRE, l1p, chunk);
  cudaError_t e = cudaFuncSetAttribute(k_count_bitslice<TW, KRE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_count_bitslice<TW, KRE><<<grid, BS_THREADS, smem, s>>>(L, V, l1p, chunk, vw);
  return cudaGetLastError();
}

template <int TW>
static cudaError_t go_k(Lattice L, const uint32_t *V, int kre, uint32_t l1p, uint32_t chunk,
                        uint64_t vw, int grid, cudaStream_t s) {
  switch (kre) {
    case 2: return go<TW, 2>(L, V, l1p, chunk, vw, grid, s);
    case 4: return go<TW, 4>(L, V, l1p, chunk, vw, grid, s);
    case 8: return go<TW, 8>(L, V, l1p, chunk, vw, grid, s);
    default: return go<TW, 16>(L, V, l1p, chunk, vw, grid, s);
  }
}

cudaError_t launch_count_bitslice(Lattice L, const uint32_t *V, int tw, int kre, uint32_t l1p,
                                  uint32_t chunk, uint64_t vwords, int grid, cudaStream_t s) {
  if (tw != 16 && tw != 8 && tw != 4) return cudaErrorInvalidValue;
  if (bitslice_tile_words(tw, l1p) % 4) return cudaErrorInvalidValue;
  switch (tw) {
    case 16: return go_k<16>(L, V, kre, l1p, chunk, vwords, grid, s);
    case 8: return go_k<8>(L, V, kre, l1p, chunk, vwords, grid, s);
    default: return go_k<4>(L, V, kre, l1p, chunk, vwords, grid, s);
  }
}

}  // namespace dic
