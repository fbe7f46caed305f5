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
//   k_gram_operand  the stop's block as an e4m3 0/1 matrix X (1.0 = 0x38),
//                   ranks x rows, in the K-major no-swizzle core-matrix
//                   layout of tcgen05 (8 rows x 16 bytes per core matrix),
//                   one contiguous 16 KiB block per (128-rank tile, 128-row
//                   chunk)
//   k_gram_pairs    one CTA per (tile pair i <= j, K split): a 4-stage ring
//                   of bulk copies (cp.async.bulk + mbarrier) feeds
//                   tcgen05.mma.kind::f8f6f4 (M = N = 128, K = 32 per
//                   instruction, fp32 accumulation in TMEM); tcgen05.ld
//                   brings each thread one row of the 128x128 tile; the
//                   rows are turned through shared memory so that the
//                   counts of pairs a < b are added to 32 consecutive
//                   records per warp instruction.
//
// Exactness: every product is 0 or 1 and a tile's sum over one split is at
// most its rows (< 2^24), so fp32 accumulation is exact.
//
// Every wait on an mbarrier is bounded; a wait that gives up records
// DIC_ETIMEOUT in the loop state, lets the copies already issued land, frees
// the tensor memory and returns.
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"
#include "lattice_device.cuh"

namespace dic {

constexpr uint32_t GT = 128;             // ranks per tile (M = N)
constexpr uint32_t GK = 128;             // rows (K) per chunk = bytes per row of a tile
constexpr uint32_t GSTAGES = 4;
constexpr uint32_t GTILE_BYTES = GT * GK;  // 16 KiB
constexpr uint32_t GRAM_THREADS = 128;
constexpr long long WAIT_CYCLES = 2000000000ll;  // ~1 s at 2 GHz before giving up
constexpr uint8_t E4M3_ONE = 0x38;

// ------------------------------------------------------------ operand X
// Byte offset of element (rank r, row k) inside its 16 KiB tile block:
// core matrix (r/8, k/16) at (r/8)*1024 + (k/16)*128, element (r%8)*16 + k%16.
__device__ __forceinline__ uint32_t core_offset(uint32_t r, uint32_t k) {
  return (r >> 3) * 1024u + (k >> 4) * 128u + (r & 7u) * 16u + (k & 15u);
}

// X block for (rank tile ti, chunk kc) starts at ((ti * nkc) + kc) * 16 KiB.
// The BITSLICE count that follows in the same stop checks (and may stall
// on) the kernel width and the box-set room before changing anything; the
// pair-cohort kernels make the same checks and do nothing when that count
// will stall, so a stop re-run after a stall never counts its pairs twice.
__device__ __forceinline__ bool gram_may_run(const Lattice &L, const Ctrl *C, uint32_t kre) {
  if (C->stall || C->done) return false;
  if (C->max_k > kre) return false;
  if ((uint64_t)(C->hash_used + C->n_live) * 2 > L.hcap) return false;
  return C->step <= L.stop_max && C->head == 0;  // the pair cohort is in DASHED
}

__global__ void __launch_bounds__(256) k_gram_operand(Lattice L, uint8_t *__restrict__ X,
                                                      uint32_t nkc_max, uint64_t xbytes,
                                                      uint32_t kre) {
  Ctrl *C = L.ctrl;
  if (!gram_may_run(L, C, kre)) return;
  const uint32_t g = C->step;
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  const uint32_t nrows = (uint32_t)(last - first);
  if (blockIdx.x == 0 && threadIdx.x == 0) C->gram_rows += nrows;
  const uint32_t nkc = (nrows + GK - 1) / GK;
  const uint32_t ngroups = nkc * (GK / 32);  // 32-row groups, incl. zero padding
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t items = (uint64_t)ngroups * L.wc;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t it = (uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < items;
       it += nwarps) {
    const uint32_t grp = (uint32_t)(it / L.wc), j = (uint32_t)(it % L.wc);
    const uint32_t t = grp * 32 + lane;
    const uint64_t x = t < nrows ? __ldg(L.rows + (first + t) * L.wc + j) : 0ull;
    const uint32_t lo = warp_transpose32((uint32_t)x);
    const uint32_t hi = warp_transpose32((uint32_t)(x >> 32));
    // lane handles ranks r0 = 64j + lane and r1 = r0 + 32: 32 rows each
    const uint32_t kc = (grp * 32) / GK, k0 = (grp * 32) % GK;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t r = j * 64 + lane + 32 * h;
      const uint32_t bits = h ? hi : lo;
      const uint32_t ti = r / GT, rr = r % GT;
      const uint64_t base = ((uint64_t)ti * nkc_max + kc) * GTILE_BYTES;
#pragma unroll
      for (int part = 0; part < 2; ++part) {  // rows k0+16*part .. +15
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const uint32_t nib = (bits >> (16 * part + 4 * q)) & 0xFu;
          w[q] = ((nib & 1u) ? (uint32_t)E4M3_ONE : 0u) |
                 ((nib & 2u) ? (uint32_t)E4M3_ONE << 8 : 0u) |
                 ((nib & 4u) ? (uint32_t)E4M3_ONE << 16 : 0u) |
                 ((nib & 8u) ? (uint32_t)E4M3_ONE << 24 : 0u);
        }
        const uint64_t off = base + core_offset(rr, k0 + 16 * part);
        if (off + 16 > xbytes) {  // internal sizing error: record, skip
          C->error = DIC_INTERNAL_BOUNDS;
          continue;
        }
        *reinterpret_cast<uint4 *>(X + off) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
  }
}

// ---------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t sm_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(bar)),
               "r"(bytes)
               : "memory");
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
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(sm_addr(dst)), "l"(src), "r"(bytes), "r"(sm_addr(bar))
      : "memory");
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

__device__ __forceinline__ uint64_t gram_pair_index(uint64_t a, uint64_t b, uint64_t l1) {
  return a * (2 * l1 - a - 1) / 2 + (b - a - 1);
}

// ------------------------------------------------------------------ GEMM
__global__ void __launch_bounds__(GRAM_THREADS, 1) k_gram_pairs(Lattice L,
                                                                const uint8_t *__restrict__ X,
                                                                uint32_t ntile, uint32_t nkc_max,
                                                                uint32_t nsplit, uint32_t kre) {
  extern __shared__ __align__(1024) uint8_t gsm[];
  __shared__ __align__(8) uint64_t full[GSTAGES], empty[GSTAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ uint32_t failed;
  Ctrl *C = L.ctrl;
  if (!gram_may_run(L, C, kre)) return;
  const uint32_t g = C->step;
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  const uint32_t nkc = (uint32_t)((last - first + GK - 1) / GK);
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
    for (uint32_t s = 0; s < GSTAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(&done, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {  // tensor memory: 128 columns of 128 lanes (fp32 accumulators)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;"
                 ::"r"(sm_addr(&tmem_base)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  const uint8_t *XA = X + ((uint64_t)ti * nkc_max) * GTILE_BYTES;
  const uint8_t *XB = X + ((uint64_t)tj * nkc_max) * GTILE_BYTES;
  uint32_t issued = 0;  // stages handed to the copy engine by the producer

  if (threadIdx.x == 0) {
    // producer: bulk copies of the A and B tiles of each K chunk
    for (uint32_t i = 0; i < nk; ++i) {
      const uint32_t s = i % GSTAGES, use = i / GSTAGES;
      if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1)) { failed = 1; break; }
      mbar_expect_tx(&full[s], 2 * GTILE_BYTES);
      bulk_g2s(stage_a + s * GTILE_BYTES, XA + (uint64_t)(kc0 + i) * GTILE_BYTES, GTILE_BYTES,
               &full[s]);
      bulk_g2s(stage_b + s * GTILE_BYTES, XB + (uint64_t)(kc0 + i) * GTILE_BYTES, GTILE_BYTES,
               &full[s]);
      ++issued;
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer: 4 instructions (K = 32 bytes each) per 128-row chunk
    for (uint32_t i = 0; i < nk; ++i) {
      const uint32_t s = i % GSTAGES, use = i / GSTAGES;
      if (!mbar_wait(&full[s], use & 1)) { failed = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = sm_addr(stage_a + s * GTILE_BYTES);
      const uint32_t b0 = sm_addr(stage_b + s * GTILE_BYTES);
#pragma unroll
      for (uint32_t q = 0; q < GK / 32; ++q)
        mma_f8(tmem, smem_desc(a0 + q * 256, 128, 1024), smem_desc(b0 + q * 256, 128, 1024),
               (i | q) != 0);
      mma_commit(&empty[s]);
    }
    mma_commit(&done);
  }
  // epilogue: every warp reads its 32 TMEM lanes (rows ti*128 + 32w + lane)
  bool ok = mbar_wait(&done, 0);
  __syncthreads();
  ok = ok && !failed;
  if (threadIdx.x == 0 && !ok) C->error = 5;  // DIC_ETIMEOUT
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // Each warp stages its 32 x 32 sub-tiles through shared memory (the
    // operand ring is idle once `done` has fired) so that a warp's adds go
    // to 32 consecutive counters: lane q adds count (a, b0 + q) of row a.
    const uint64_t l1 = L.l1;
    uint32_t *stage = reinterpret_cast<uint32_t *>(stage_a) + warp * (32 * 33);
    const uint64_t a0 = (uint64_t)ti * GT + warp * 32;
    for (uint32_t c0 = 0; c0 < GT; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((warp * 32u) << 16) + c0;
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
      if (a0 >= l1 || (uint64_t)tj * GT + c0 + 31 <= a0) continue;  // all b <= a (warp-uniform)
#pragma unroll
      for (int q = 0; q < 32; ++q) stage[lane * 33 + q] = (uint32_t)__uint_as_float(v[q]);
      __syncwarp();
      const uint32_t rmax = l1 - a0 < 32 ? (uint32_t)(l1 - a0) : 32u;
      for (uint32_t r = 0; r < rmax; ++r) {
        const uint64_t a = a0 + r;
        const uint32_t cnt = stage[r * 33 + lane];
        if (b > a && b < l1 && cnt) atomicAdd(&L.csupp[gram_pair_index(a, b, l1)], cnt);
      }
      __syncwarp();
    }
  } else if (threadIdx.x == 0) {
    // let the copies already issued land before the shared memory goes away
    for (uint32_t i = (issued > GSTAGES ? issued - GSTAGES : 0); i < issued; ++i)
      mbar_wait(&full[i % GSTAGES], (i / GSTAGES) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

// -------------------------------------------------------------- launchers
uint32_t gram_tiles(uint32_t l1) { return (l1 + GT - 1) / GT; }
uint32_t gram_chunks(uint64_t rows) { return (uint32_t)((rows + GK - 1) / GK); }
uint64_t gram_operand_bytes(uint32_t l1, uint64_t block_rows) {
  return (uint64_t)gram_tiles(l1) * gram_chunks(block_rows) * GTILE_BYTES;
}

cudaError_t launch_gram_operand(Lattice L, uint8_t *X, uint32_t nkc_max, uint64_t xbytes,
                                uint32_t kre, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t items = (uint64_t)nkc_max * (GK / 32) * L.wc;
  uint64_t want = (items + 7) / 8;
  int grid = (int)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
  if (grid < 1) grid = 1;
  k_gram_operand<<<grid, 256, 0, s>>>(L, X, nkc_max, xbytes, kre);
  return cudaGetLastError();
}

cudaError_t launch_gram_pairs(Lattice L, const uint8_t *X, uint32_t nkc_max, uint32_t nsplit,
                              uint32_t kre, cudaStream_t s) {
  const uint32_t ntile = gram_tiles(L.l1);
  const uint32_t npair_tiles = ntile * (ntile + 1) / 2;
  // two rings of tiles + a 16 KiB guard band after them
  const size_t smem = 2 * GSTAGES * GTILE_BYTES + GTILE_BYTES;
  cudaError_t e =
      cudaFuncSetAttribute(k_gram_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gram_pairs<<<npair_tiles * nsplit, GRAM_THREADS, smem, s>>>(L, X, ntile, nkc_max, nsplit,
                                                                 kre);
  return cudaGetLastError();
}

}  // namespace dic
