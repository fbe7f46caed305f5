// Measured integer-ALU issue rate: the denominator of the BITSLICE count's
// roofline (its algorithmic work is one AND per rank word, one popcount and
// one add per 32-row word). Eight independent chains of 3-input logic ops
// (lop3.b32, the instruction an AND of column words compiles to) per thread,
// every SM filled, timed with CUDA events.
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"

namespace dic {

constexpr int ALU_CHAINS = 8;
constexpr int ALU_UNROLL = 16;
constexpr int ALU_THREADS = 256;

__device__ __forceinline__ uint32_t lop3_xor3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__global__ void __launch_bounds__(ALU_THREADS) k_alu_peak(uint32_t *out, uint32_t iters,
                                                          uint32_t seed) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[ALU_CHAINS];
#pragma unroll
  for (int c = 0; c < ALU_CHAINS; ++c) x[c] = seed * (t + 1) + 0x9E3779B9u * (c + 1);
  const uint32_t b = seed ^ t, d = ~seed + t;
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < ALU_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < ALU_CHAINS; ++c) x[c] = lop3_xor3(x[c], b, d);
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < ALU_CHAINS; ++c) r ^= x[c];
  out[t] = r;  // keeps the chains live
}

// Tera lop3 ops per second over one launch of a few ms after a warm-up launch.
cudaError_t measure_alu_peak(double *tops) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint32_t blocks = (uint32_t)sms * 8;  // 2,048 threads per SM
  const uint64_t threads = (uint64_t)blocks * ALU_THREADS;
  uint32_t *out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaMalloc(&out, threads * 4);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  const uint32_t iters = 2048;  // 2048 x 16 x 8 = 262,144 ops per thread
  float ms = 0;
  if (e == cudaSuccess) {
    k_alu_peak<<<blocks, ALU_THREADS, 0, s>>>(out, 64, 12345u);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) {
    k_alu_peak<<<blocks, ALU_THREADS, 0, s>>>(out, iters, 54321u);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (e == cudaSuccess && ms > 0)
    *tops = (double)threads * iters * ALU_UNROLL * ALU_CHAINS / (ms * 1e-3) / 1e12;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  return e;
}

}  // namespace dic
