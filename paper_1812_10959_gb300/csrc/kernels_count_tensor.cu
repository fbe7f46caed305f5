// COUNTSUPPORT (Algorithm 3) for the pair cohort on the tensor cores.
//
// For a 2-itemset {a, b} the containment test (T AND C) == C is T[a]*T[b] =
// 1, so the supports of ALL pairs over a block are the Gram matrix of the
// block's 0/1 item columns: supp(a, b) = sum_t X[a][t] * X[b][t], a dense
// contraction over the block's rows. The first-pass pair join makes the pair
// cohort exactly "all pairs a < b of frequent ranks" in lexicographic order,
// so pair {a, b} is record pair_off(a) + b - a - 1 and the GEMM's output
// element (a, b) goes straight to its counter.
//
// k_gram_pairs: one CTA per (128-rank tile pair i <= j, K split). The
// operands come from the stop's bit columns V (the BITSLICE transposition,
// 32 rows per word): for every 128-row chunk, sixteen expander warps load
// each rank's four column words (a few chunks ahead) and write them to
// shared memory as e4m3 0/1 bytes (1.0 = 0x38) in the K-major no-swizzle
// core-matrix layout of tcgen05 (8 ranks x 16 rows per 128-byte core
// matrix), through a 4-stage ring guarded by mbarriers; one thread of a
// seventeenth warp issues
// tcgen05.mma.kind::f8f6f4 (M = N = 128, K = 32 per instruction, fp32
// accumulation in tensor memory). The epilogue brings the 128x128 tile out
// with tcgen05.ld, turns its rows through shared memory and adds the counts
// of pairs a < b to 32 consecutive records per warp instruction.
//
// Exactness: every product is 0 or 1 and a tile's sum over one split is at
// most its rows (< 2^24), so fp32 accumulation is exact.
//
// Every wait on an mbarrier is bounded; a wait that gives up records
// DIC_ETIMEOUT in the loop state, lets the tensor instructions already
// issued finish, frees the tensor memory and returns.
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"
#include "lattice_device.cuh"

namespace dic {

constexpr uint32_t GT = 128;             // ranks per tile (M = N)
constexpr uint32_t GK = 128;             // rows (K) per chunk = bytes per row of a tile
constexpr uint32_t GSTAGES = 4;
constexpr uint32_t GTILE_BYTES = GT * GK;  // 16 KiB
constexpr uint32_t GEXP_WARPS = 16;      // expander / epilogue warps
constexpr uint32_t GPREFETCH = 4;        // chunks of column words loaded ahead
constexpr uint32_t GEXP_THREADS = GEXP_WARPS * 32;
constexpr uint32_t GRAM_THREADS = GEXP_THREADS + 32;  // + the MMA warp
constexpr long long WAIT_CYCLES = 2000000000ll;  // ~1 s at 2 GHz before giving up
constexpr uint8_t E4M3_ONE = 0x38;

// Byte offset of element (rank r, row k) inside a 16 KiB tile: core matrix
// (r/8, k/16) at (r/8)*1024 + (k/16)*128, element (r%8)*16 + k%16.
__device__ __forceinline__ uint32_t core_offset(uint32_t r, uint32_t k) {
  return (r >> 3) * 1024u + (k >> 4) * 128u + (r & 7u) * 16u + (k & 15u);
}

// Four 0/1 bits -> four bytes of 0 or e4m3 1.0: the multiply places bit q at
// bit 8q (its other copies land on bits the mask clears; no carries).
__device__ __forceinline__ uint32_t expand4(uint32_t nib) {
  return ((nib * 0x00204081u) & 0x01010101u) * (uint32_t)E4M3_ONE;
}

// ---------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t sm_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(sm_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait (about a second of SM clock); false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (clock64() - t0 < WAIT_CYCLES)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Generic-proxy shared-memory writes -> visible to the tensor core's reads.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Shared-memory operand descriptor: K-major, no swizzle; leading byte offset
// = distance between core matrices along K, stride byte offset = distance
// between 8-row groups; bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// Instruction descriptor, kind::f8f6f4: D f32 (bits 4-5 = 1), A and B e4m3
// (0), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t GRAM_IDESC = (1u << 4) | ((GT >> 3) << 17) | ((GT >> 4) << 24);

__device__ __forceinline__ void mma_f8(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem), "l"(a), "l"(b), "r"(GRAM_IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
      ::"r"(sm_addr(bar))
      : "memory");
}


// ------------------------------------------------------------------ GEMM
// Expand 32 rows of one rank's column (bit j of w = row 32 q0 + j of the
// chunk) into the tile at rank row rr (arithmetic only: no shared-memory
// reads beside the tensor core's).
__device__ __forceinline__ void expand_rows32(uint8_t *tile, uint32_t rr, uint32_t q0,
                                              uint32_t w) {
#pragma unroll
  for (uint32_t h = 0; h < 2; ++h) {  // 16 rows each
    const uint32_t x = w >> (16 * h);
    *reinterpret_cast<uint4 *>(tile + core_offset(rr, 32 * q0 + 16 * h)) =
        make_uint4(expand4(x & 0xFu), expand4((x >> 4) & 0xFu), expand4((x >> 8) & 0xFu),
                   expand4((x >> 12) & 0xFu));
  }
}

__global__ void __launch_bounds__(GRAM_THREADS, 1) k_gram_pairs(Lattice L, uint32_t ntile,
                                                                uint32_t nsplit, uint32_t kre) {
  extern __shared__ __align__(1024) uint8_t gsm[];
  __shared__ __align__(8) uint64_t full[GSTAGES], empty[GSTAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile uint32_t failed;
  Ctrl *C = L.ctrl;
  if (!gram_may_run(L, C, kre)) return;
  const uint32_t g = C->step;
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  const uint32_t nrows = (uint32_t)(last - first);
  if (blockIdx.x == 0 && threadIdx.x == 0) C->gram_rows += nrows;
  const uint32_t nkc = (nrows + GK - 1) / GK;
  // which tile pair (ti <= tj) and which K split
  const uint32_t pair = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
  uint32_t ti = 0, rem = pair;
  while (ti < ntile && rem >= ntile - ti) { rem -= ntile - ti; ++ti; }
  if (ti >= ntile) return;
  const uint32_t tj = ti + rem;
  const uint32_t per = (nkc + nsplit - 1) / nsplit;
  const uint32_t kc0 = split * per;
  const uint32_t kc1 = kc0 + per < nkc ? kc0 + per : nkc;
  if (kc0 >= kc1) return;  // nothing to count for this split (uniform per CTA)
  const uint32_t nk = kc1 - kc0;
  uint8_t *stage_a = gsm;                          // GSTAGES x 16 KiB
  uint8_t *stage_b = gsm + GSTAGES * GTILE_BYTES;  // GSTAGES x 16 KiB
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < GSTAGES; ++s) {
      mbar_init(&full[s], GEXP_WARPS);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == GEXP_WARPS) {  // tensor memory: 128 columns of 128 lanes (fp32)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;"
                 ::"r"(sm_addr(&tmem_base)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp < GEXP_WARPS) {
    // expanders: thread (rank rr, quarter q0) writes rows [32 q0, 32 q0 + 32)
    // of rank rr of both tiles for every chunk; the column words of the next
    // GPREFETCH chunks are in flight while a chunk is expanded
    const uint32_t rr = threadIdx.x % GT, q0 = threadIdx.x / GT;
    const uint64_t ra = (uint64_t)ti * GT + rr, rb = (uint64_t)tj * GT + rr;
    const bool oka = ra < L.l1, okb = rb < L.l1;
    const uint32_t tw = L.tw, st = bs_stride((int)tw), l1p = L.l1p;
    const uint32_t tw_shift = __ffs(tw) - 1;  // tw is 4, 8 or 16
    const uint32_t *__restrict__ V = L.V;
    auto load = [&](uint32_t kc, uint64_t r, bool ok) -> uint32_t {
      const uint32_t w0 = kc * (GK / 32) + q0;  // 32-row word of this quarter
      const uint64_t t = w0 >> tw_shift, wi = w0 & (tw - 1);
      return ok ? __ldg(V + (t * l1p + r) * st + wi) : 0u;
    };
    uint32_t qa[GPREFETCH], qb[GPREFETCH];
#pragma unroll
    for (uint32_t u = 0; u < GPREFETCH; ++u) {
      qa[u] = u < nk ? load(kc0 + u, ra, oka) : 0u;
      qb[u] = u < nk ? load(kc0 + u, rb, okb) : 0u;
    }
    for (uint32_t i0 = 0; i0 < nk; i0 += GPREFETCH) {
#pragma unroll
      for (uint32_t u = 0; u < GPREFETCH; ++u) {
        const uint32_t i = i0 + u;
        if (i >= nk || __shfl_sync(0xffffffffu, failed, 0)) break;  // warp-uniform
        const uint32_t s = i % GSTAGES, use = i / GSTAGES;
        const uint32_t wa = qa[u], wb = qb[u];
        if (i + GPREFETCH < nk) {
          qa[u] = load(kc0 + i + GPREFETCH, ra, oka);
          qb[u] = load(kc0 + i + GPREFETCH, rb, okb);
        }
        // one lane per warp waits for the ring slot and one arrives for the
        // warp (the barrier counts warps, not threads)
        bool slot_ok = true;
        if (use > 0 && lane == 0) slot_ok = mbar_wait(&empty[s], (use - 1) & 1);
        if (!__shfl_sync(0xffffffffu, slot_ok ? 1u : 0u, 0)) { failed = 1; break; }
        expand_rows32(stage_a + s * GTILE_BYTES, rr, q0, wa);
        expand_rows32(stage_b + s * GTILE_BYTES, rr, q0, wb);
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[s]);
      }
    }
  } else if (lane == 0) {
    // MMA issuer: 4 instructions (K = 32 bytes each) per 128-row chunk
    for (uint32_t i = 0; i < nk; ++i) {
      const uint32_t s = i % GSTAGES, use = i / GSTAGES;
      if (failed || !mbar_wait(&full[s], use & 1)) { failed = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = sm_addr(stage_a + s * GTILE_BYTES);
      const uint32_t b0 = sm_addr(stage_b + s * GTILE_BYTES);
#pragma unroll
      for (uint32_t q = 0; q < GK / 32; ++q)
        mma_f8(tmem, smem_desc(a0 + q * 256, 128, 1024), smem_desc(b0 + q * 256, 128, 1024),
               (i | q) != 0);
      mma_commit(&empty[s]);
    }
    mma_commit(&done);  // arrives once every MMA issued above has completed
  }
  __syncwarp();
  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (ranks of tile ti),
  // columns 32 (w / 4) .. +31
  if (lane == 0 && !mbar_wait(&done, 0)) failed = 1;
  __syncthreads();
  const bool ok = !failed;  // the same for every thread of the CTA
  if (threadIdx.x == 0 && !ok) C->error = 5;  // DIC_ETIMEOUT
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && warp < GEXP_WARPS) {
    // Each warp stages its 32 x 32 sub-tile through shared memory (the
    // operand rings, 128 KiB, are idle once `done` has fired) so that a
    // warp's adds go to 32 consecutive counters: lane q adds count (a, b0 + q)
    // of row a.
    const uint64_t l1 = L.l1;
    uint32_t *stage = reinterpret_cast<uint32_t *>(stage_a) + warp * (32 * 33);
    const uint32_t lq = warp % 4;
    const uint64_t a0 = (uint64_t)ti * GT + lq * 32;
    do {
      const uint32_t c0 = (warp / 4) * 32;
      uint32_t v[32];
      const uint32_t taddr = tmem + ((lq * 32u) << 16) + c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
          "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const uint64_t b = (uint64_t)tj * GT + c0 + lane;
      if (a0 >= l1 || (uint64_t)tj * GT + c0 + 31 <= a0) break;  // all b <= a (warp-uniform)
#pragma unroll
      for (int q = 0; q < 32; ++q) stage[lane * 33 + q] = (uint32_t)__uint_as_float(v[q]);
      __syncwarp();
      const uint32_t rmax = l1 - a0 < 32 ? (uint32_t)(l1 - a0) : 32u;
      for (uint32_t r = 0; r < rmax; ++r) {
        const uint64_t a = a0 + r;
        const uint32_t cnt = stage[r * 33 + lane];
        if (b > a && b < l1 && cnt) atomicAdd(&L.csupp[pair_record(a, b, l1)], cnt);
      }
    } while (0);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == GEXP_WARPS)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

// -------------------------------------------------------------- launchers
uint32_t gram_tiles(uint32_t l1) { return (l1 + GT - 1) / GT; }
uint32_t gram_chunks(uint64_t rows) { return (uint32_t)((rows + GK - 1) / GK); }

cudaError_t launch_gram_pairs(Lattice L, uint32_t nsplit, uint32_t kre, cudaStream_t s) {
  const uint32_t ntile = gram_tiles(L.l1);
  const uint32_t npair_tiles = ntile * (ntile + 1) / 2;
  const size_t smem = 2 * GSTAGES * GTILE_BYTES;  // the A and B rings
  cudaError_t e =
      cudaFuncSetAttribute(k_gram_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_pairs<<<npair_tiles * nsplit, GRAM_THREADS, smem, s>>>(L, ntile, nsplit, kre);
  return cudaGetLastError();
}

}  // namespace dic
