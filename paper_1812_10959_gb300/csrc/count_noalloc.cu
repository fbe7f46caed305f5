// dic_count_support_noalloc: support counting that never allocates memory.
//
// Who needs this: callers that are not allowed to call cudaMalloc (or any
// allocator) at the point where they need supports counted -- for example
// code running inside a memory-capped or pre-reserved allocation regime, a
// host thread that must not take the driver's allocation locks, or an
// embedding runtime that owns all device memory itself. Every other entry
// point of this library allocates its working buffers per call; this one
// keeps its working buffer in a file-scope __device__ array instead.
//
// What it computes: for each candidate itemset C (a bitmask of W = ceil(m/64)
// words, item p in bit p%64 of word p/64) the number of rows T of a
// device-resident bitmap database with (T AND C) == C. Rows are processed in
// slabs: a slab is transposed into one bit column per item (32 rows per
// 32-bit word) in the static scratch array, then every candidate's count over
// the slab is the popcount of the AND of its items' columns.
//
// Scratch: g_noalloc_cols, DIC_NOALLOC_SCRATCH_WORDS 32-bit words (4 MiB),
// resident on every device that loads this library until the process exits.
// All calls share it and it keeps the last call's contents; nothing in it
// needs to start at zero (every word a call reads is written earlier in the
// same call). Calls whose GPU work overlaps (different streams, or different
// host threads on the same device) race on it and give wrong counts: order
// them on one stream or serialise them.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/dic.h"
#include "dic_internal.cuh"

namespace {

constexpr uint32_t kScratchWords = DIC_NOALLOC_SCRATCH_WORDS;
constexpr uint32_t kMaxItems = DIC_NOALLOC_MAX_ITEMS;
constexpr uint32_t kMaxDevices = 64;

__device__ __align__(256) uint32_t g_noalloc_cols[kScratchWords];

// Device address of g_noalloc_cols, looked up once per device (host code may
// not use the symbol itself: on the host it names a stand-in, not device
// memory).
std::mutex g_setup_mu;
uint32_t *g_cols_addr[kMaxDevices] = {nullptr};

dic_status noalloc_fail(dic_status s, const char *msg) {
  dic::set_last_error(msg);
  return s;
}

// cols[i * vw + w], bit j = row r0 + 32w + j contains item i; w < nw.
__global__ void k_noalloc_slice(const uint64_t *__restrict__ words, uint32_t W, uint32_t m,
                                uint64_t r0, uint32_t nrows, uint32_t *__restrict__ cols,
                                uint32_t vw) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nw = (nrows + 31) / 32;
  const uint64_t items = (uint64_t)nw * W;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t it = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items;
       it += nwarps) {
    const uint32_t w = (uint32_t)(it / W), j = (uint32_t)(it % W);
    const uint32_t rr = 32 * w + lane;
    const uint64_t x = rr < nrows ? __ldg(words + (r0 + rr) * W + j) : 0ull;
    uint32_t lo = 0, hi = 0;
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      const uint32_t v = __ballot_sync(0xffffffffu, (uint32_t)(x >> b) & 1u);
      if ((int)lane == b) lo = v;
    }
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      const uint32_t v = __ballot_sync(0xffffffffu, (uint32_t)(x >> (b + 32)) & 1u);
      if ((int)lane == b) hi = v;
    }
    const uint32_t i0 = j * 64 + lane, i1 = i0 + 32;
    if (i0 < m) cols[(uint64_t)i0 * vw + w] = lo;
    if (i1 < m) cols[(uint64_t)i1 * vw + w] = hi;
  }
}

// supp[c] += rows of the slab containing masks[c]: one warp per candidate,
// its lanes on consecutive 32-row column words (coalesced loads of each
// item's column), the lanes' popcounts summed across the warp.
__global__ void k_noalloc_count(const uint64_t *__restrict__ masks, uint32_t ncand, uint32_t W,
                                uint32_t m, const uint32_t *__restrict__ cols, uint32_t vw,
                                uint32_t nrows, uint32_t *__restrict__ supp) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t nw = (nrows + 31) / 32;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < ncand;
       c += nwarps) {
    const uint64_t *mk = masks + c * W;
    uint32_t cnt = 0;
    for (uint32_t w = lane; w < nw; w += 32) {
      // rows of the slab that exist: all 32 bits except in the last word
      uint32_t acc = w + 1 < nw || nrows % 32 == 0 ? 0xffffffffu : (1u << (nrows % 32)) - 1u;
      for (uint32_t j = 0; j < W && acc; ++j) {
        for (uint64_t x = __ldg(mk + j); x; x &= x - 1) {
          const uint32_t item = j * 64 + (uint32_t)(__ffsll((long long)x) - 1);
          if (item >= m) {  // no row holds an item >= m
            acc = 0;
            break;
          }
          acc &= __ldg(cols + (uint64_t)item * vw + w);
        }
      }
      cnt += __popc(acc);
    }
    cnt = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) supp[c] += cnt;
  }
}

}  // namespace

extern "C" dic_status dic_count_support_noalloc(const uint64_t *dev_words, uint64_t n, uint32_t m,
                                                const uint64_t *dev_masks, uint32_t ncand,
                                                uint32_t *dev_supp, void *stream) {
  if (m == 0 || m > kMaxItems)
    return noalloc_fail(DIC_EINVAL, "dic_count_support_noalloc: m must be in 1..4096");
  if (n >= (1ull << 31)) return noalloc_fail(DIC_EINVAL, "dic_count_support_noalloc: n >= 2^31");
  if (ncand == 0) return DIC_OK;
  if (!dev_supp || !dev_masks || (n && !dev_words))
    return noalloc_fail(DIC_EINVAL, "dic_count_support_noalloc: NULL buffer");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= (int)kMaxDevices)
    return noalloc_fail(DIC_ECUDA, "dic_count_support_noalloc: no usable current device");
  uint32_t *cols = nullptr;
  {
    // first call on this device: resolve the scratch array's device address
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_cols_addr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_cols);
      if (e != cudaSuccess || !p)
        return noalloc_fail(DIC_ECUDA, "dic_count_support_noalloc: cudaGetSymbolAddress failed");
      g_cols_addr[dev] = static_cast<uint32_t *>(p);
    }
    cols = g_cols_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t W = (m + 63) / 64;
  // slab height: as many 32-row words per item column as the scratch holds
  uint32_t vw = kScratchWords / m;
  if (vw > 2048) vw = 2048;
  const uint64_t slab = (uint64_t)vw * 32;
  if (cudaMemsetAsync(dev_supp, 0, (size_t)ncand * 4, s) != cudaSuccess)
    return noalloc_fail(DIC_ECUDA, "dic_count_support_noalloc: clearing the counts failed");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  // each launch's own status (cudaLaunchKernelEx), so an error left over
  // from unrelated earlier work is neither reported here nor cleared
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(256);
  cfg.stream = s;
  for (uint64_t r0 = 0; r0 < n; r0 += slab) {
    const uint32_t nrows = (uint32_t)(n - r0 < slab ? n - r0 : slab);
    const uint64_t sitems = (uint64_t)((nrows + 31) / 32) * W;
    int g1 = (int)((sitems + 7) / 8 < (uint64_t)sms * 8 ? (sitems + 7) / 8 : (uint64_t)sms * 8);
    cfg.gridDim = dim3(g1 > 0 ? g1 : 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_noalloc_slice, dev_words, W, m, r0, nrows, cols, vw);
    if (e != cudaSuccess)
      return noalloc_fail(DIC_ECUDA, "dic_count_support_noalloc: slice launch failed");
    // one warp per candidate, eight per CTA
    int g2 = (int)((ncand + 7) / 8 < (uint32_t)sms * 8 ? (ncand + 7) / 8 : sms * 8);
    cfg.gridDim = dim3(g2);
    e = cudaLaunchKernelEx(&cfg, k_noalloc_count, dev_masks, ncand, W, m,
                           (const uint32_t *)cols, vw, nrows, dev_supp);
    if (e != cudaSuccess)
      return noalloc_fail(DIC_ECUDA, "dic_count_support_noalloc: count launch failed");
  }
  return DIC_OK;
}
