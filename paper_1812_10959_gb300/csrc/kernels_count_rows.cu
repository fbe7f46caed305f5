// COUNTSUPPORT (Algorithm 3), ROWS path: the containment test of Section
// 4.1, (BitMask(T) AND BitMask(C)) == BitMask(C), on row-major bitmaps.
//
// Mapping (the loop interchange of Figure 2): one thread owns one candidate
// and walks the block's rows, so each count lives in one register and no two
// threads ever update the same counter within a tile. A candidate of k items
// touches at most k of the row's 32-bit halves; the thread keeps only those
// (index, mask) pairs in registers and tests
//     acc = OR_h (mask_h AND NOT row[idx_h]);   contained <=> acc == 0
// (one LOP3 per half). Rows are staged through shared memory in chunks and
// read as broadcasts (all lanes read the same row).
//
// Load balance (Figure 3): when there are few candidates the block's rows are
// split across CTAs as well and partial counts are merged with atomicAdd,
// the GPU form of the nested reduction(+) of Algorithm 3.
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"

namespace dic {

constexpr int ROWS_THREADS = 256;

template <int NW>
__global__ void __launch_bounds__(ROWS_THREADS) k_count_rows(Lattice L, uint32_t rch) {
  extern __shared__ uint32_t srow[];
  pdl_wait();
  pdl_trigger();
  Ctrl *C = L.ctrl;
  if (C->stall || C->done) return;
  const uint32_t wc = L.wc, hw = 2 * wc;
  {
    const uint32_t need = C->max_k < hw ? C->max_k : hw;
    if (need > (uint32_t)NW) {
      if (blockIdx.x == 0 && threadIdx.x == 0) C->stall = ST_WIDTH;
      return;
    }
  }
  const uint32_t g = C->step, tail = C->tail;
  // (the pair cohort is skipped while its outcome is precomputed)
  const uint32_t head = counted_lo(L, C->head, tail, g, false);
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  const uint64_t nrows = last - first;
  const uint32_t ncand = tail - head;
  const uint32_t ntiles = (ncand + ROWS_THREADS - 1) / ROWS_THREADS;
  if (ntiles == 0 || nrows == 0) return;
  // rows split so that there are enough work items for the grid, each split
  // keeping at least two chunks of rows
  uint64_t nsplit = (gridDim.x + ntiles - 1) / ntiles;
  const uint64_t maxsplit = (nrows + 2 * rch - 1) / (2 * rch);
  if (nsplit > maxsplit) nsplit = maxsplit;
  if (nsplit < 1) nsplit = 1;
  const uint64_t per = (nrows + nsplit - 1) / nsplit;
  const uint64_t nwork = (uint64_t)ntiles * nsplit;

  for (uint64_t work = blockIdx.x; work < nwork; work += gridDim.x) {
    const uint32_t tile = (uint32_t)(work / nsplit);
    const uint64_t split = work % nsplit;
    const uint32_t c = head + tile * ROWS_THREADS + threadIdx.x;
    bool live = c < tail && L.cshape[c] != SH_NIL;
    // the candidate's nonzero 32-bit halves, in registers
    uint32_t idx[NW], msk[NW];
    uint32_t nw = 0;
    {
      const uint32_t *m32 = reinterpret_cast<const uint32_t *>(L.cmask + (uint64_t)c * wc);
      uint32_t h = 0;
#pragma unroll
      for (int q = 0; q < NW; ++q) {
        idx[q] = 0;
        msk[q] = 0;
        if (live) {
          while (h < hw && m32[h] == 0) ++h;
          if (h < hw) {
            idx[q] = h;
            msk[q] = m32[h];
            ++h;
            ++nw;
          }
        }
      }
    }
    uint32_t nwarp = nw;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint32_t v = __shfl_xor_sync(0xffffffffu, nwarp, o);
      nwarp = v > nwarp ? v : nwarp;
    }
    const uint64_t r0 = first + split * per;
    const uint64_t r1 = (r0 + per < last) ? r0 + per : last;
    uint32_t cnt = 0;
    for (uint64_t base = r0; base < r1; base += rch) {
      const uint32_t nr = (uint32_t)((r1 - base) < rch ? (r1 - base) : rch);
      __syncthreads();
      {
        const uint64_t *src = L.rows + base * wc;
        uint64_t *dst = reinterpret_cast<uint64_t *>(srow);
        const uint32_t nwords = nr * wc;
        for (uint32_t i = threadIdx.x; i < nwords; i += ROWS_THREADS) dst[i] = __ldg(src + i);
      }
      __syncthreads();
      if (live) {
        for (uint32_t r = 0; r < nr; ++r) {
          const uint32_t *row = srow + r * hw;
          uint32_t acc = 0;
#pragma unroll
          for (int q = 0; q < NW; ++q)
            if ((uint32_t)q < nwarp) acc |= msk[q] & ~row[idx[q]];
          cnt += acc == 0;
        }
      }
    }
    if (live && cnt) atomicAdd(&L.csupp[c], cnt);
    // algorithmic work: one LOP3 per touched half + compare + add, per test
    warp_add_u64(&C->work, live ? (unsigned long long)(nw + 2) * (r1 > r0 ? r1 - r0 : 0) : 0ull);
  }
}

// Generic width: any number of halves, mask words read from global memory.
__global__ void __launch_bounds__(ROWS_THREADS) k_count_rows_dense(Lattice L, uint32_t rch) {
  extern __shared__ uint32_t srow[];
  pdl_wait();
  pdl_trigger();
  Ctrl *C = L.ctrl;
  if (C->stall || C->done) return;
  const uint32_t wc = L.wc;
  const uint32_t g = C->step, tail = C->tail;
  const uint32_t head = counted_lo(L, C->head, tail, g, false);
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  const uint64_t nrows = last - first;
  const uint32_t ncand = tail - head;
  const uint32_t ntiles = (ncand + ROWS_THREADS - 1) / ROWS_THREADS;
  if (ntiles == 0 || nrows == 0) return;
  uint64_t nsplit = (gridDim.x + ntiles - 1) / ntiles;
  const uint64_t maxsplit = (nrows + 2 * rch - 1) / (2 * rch);
  if (nsplit > maxsplit) nsplit = maxsplit;
  if (nsplit < 1) nsplit = 1;
  const uint64_t per = (nrows + nsplit - 1) / nsplit;
  const uint64_t nwork = (uint64_t)ntiles * nsplit;
  for (uint64_t work = blockIdx.x; work < nwork; work += gridDim.x) {
    const uint32_t tile = (uint32_t)(work / nsplit);
    const uint64_t split = work % nsplit;
    const uint32_t c = head + tile * ROWS_THREADS + threadIdx.x;
    const bool live = c < tail && L.cshape[c] != SH_NIL;
    const uint64_t *mk = L.cmask + (uint64_t)c * wc;
    const uint64_t r0 = first + split * per;
    const uint64_t r1 = (r0 + per < last) ? r0 + per : last;
    uint32_t cnt = 0;
    for (uint64_t base = r0; base < r1; base += rch) {
      const uint32_t nr = (uint32_t)((r1 - base) < rch ? (r1 - base) : rch);
      __syncthreads();
      {
        const uint64_t *src = L.rows + base * wc;
        uint64_t *dst = reinterpret_cast<uint64_t *>(srow);
        for (uint32_t i = threadIdx.x; i < nr * wc; i += ROWS_THREADS) dst[i] = __ldg(src + i);
      }
      __syncthreads();
      if (live) {
        const uint64_t *rows64 = reinterpret_cast<const uint64_t *>(srow);
        for (uint32_t r = 0; r < nr; ++r) {
          uint64_t acc = 0;
          for (uint32_t w = 0; w < wc; ++w) {
            const uint64_t x = __ldg(mk + w);
            acc |= x & ~rows64[r * wc + w];
          }
          cnt += acc == 0;
        }
      }
    }
    if (live && cnt) atomicAdd(&L.csupp[c], cnt);
    warp_add_u64(&C->work,
                 live ? (unsigned long long)(2 * wc + 2) * (r1 > r0 ? r1 - r0 : 0) : 0ull);
  }
}

int rows_width_bucket(uint32_t max_k, uint32_t wc) {
  uint32_t need = max_k < 2 * wc ? max_k : 2 * wc;
  if (need <= 2) return 2;
  if (need <= 4) return 4;
  if (need <= 8) return 8;
  if (need <= 16) return 16;
  if (need <= 32) return 32;
  return 0;  // dense
}

static uint32_t rows_chunk(uint32_t wc) {
  uint32_t r = 16384u / (wc * 8u);
  if (r > 128) r = 128;
  if (r < 8) r = 8;
  return r;
}

template <int NW>
static cudaError_t go(Lattice L, int grid, uint32_t rch, size_t smem, cudaStream_t s) {
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_count_rows<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
  return launch_k(k_count_rows<NW>, grid, ROWS_THREADS, smem, s, L, rch);
}

cudaError_t launch_count_rows(Lattice L, int nw, int grid, cudaStream_t s) {
  const uint32_t rch = rows_chunk(L.wc);
  const size_t smem = (size_t)rch * L.wc * 8;
  switch (nw) {
    case 2: return go<2>(L, grid, rch, smem, s);
    case 4: return go<4>(L, grid, rch, smem, s);
    case 8: return go<8>(L, grid, rch, smem, s);
    case 16: return go<16>(L, grid, rch, smem, s);
    case 32: return go<32>(L, grid, rch, smem, s);
    default:
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_count_rows_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
      return launch_k(k_count_rows_dense, grid, ROWS_THREADS, smem, s, L, rch);
  }
}

}  // namespace dic
