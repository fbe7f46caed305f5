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
// k_gram_pairs: one CTA per (128-rank A tile i, 256-rank B tile j >= i/2,
// K split). The operands come from the stop's bit columns V (the BITSLICE
// transposition, 32 rows per word): for every 256-row chunk, twelve
// expander warps (a thread per rank row) load each rank's eight column words
// (a chunk or two ahead, two 16-byte loads) and write them to shared memory as
// e4m3 bytes (0, or 0x08 = 2^-6 for a set bit; the chunk's rows in a fixed
// order along K, the same for both operands) in the K-major no-swizzle core-matrix layout
// of tcgen05 (8 ranks x 16 rows per 128-byte core matrix), through a
// 2-stage ring guarded by mbarriers (a stage of 256 rows halves the waits,
// fences and arrivals per row of 128-row stages and gives each expander
// eight independent words); one thread of a seventeenth warp issues
// tcgen05.mma.kind::f8f6f4 (M = 128, N = 256, K = 32 per instruction, fp32
// accumulation in tensor memory). Sixteen warps then bring the 128x256 tile
// out with tcgen05.ld, turn its rows through shared memory and add the
// counts of pairs a < b to 32 consecutive records per warp instruction.
//
// Exactness: every product is 0 or 2^-12 and a tile's sum over one split is
// at most its rows (< 2^24) times 2^-12, so fp32 accumulation is exact and
// the epilogue's scaling by 2^12 returns the integer count.
//
// Every wait on an mbarrier is bounded; a wait that gives up records
// DIC_ETIMEOUT in the loop state, lets the tensor instructions already
// issued finish, frees the tensor memory and returns.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"
#include "lattice_device.cuh"

namespace dic {

constexpr uint32_t GM = 128;             // A-tile ranks (MMA M, TMEM lanes)
constexpr uint32_t GN = 256;             // B-tile ranks (MMA N, TMEM columns)
constexpr uint32_t GK = 256;             // rows (K) per chunk = bytes per rank row of a tile
constexpr uint32_t GSTAGES = 2;
constexpr uint32_t GTILE_A = GM * GK;    // 32 KiB
constexpr uint32_t GTILE_B = GN * GK;    // 64 KiB
constexpr uint32_t GQ = GK / 128;        // 16-byte column loads (four words) per rank and chunk
constexpr uint32_t GSBO = GK / 16 * 128; // bytes between 8-rank groups of a tile
constexpr uint32_t GEXP_WARPS = 16;      // epilogue warps (4 TMEM lane quarters x 4)
constexpr uint32_t GLOAD_WARPS = (GM + GN) / 32;  // expander warps: one thread per rank row
constexpr uint32_t GPREFETCH = 2;        // chunks of column words loaded ahead
constexpr uint32_t GEXP_THREADS = GEXP_WARPS * 32;
constexpr uint32_t GRAM_THREADS = GEXP_THREADS + 32;  // + the MMA warp
static_assert((GM + GN) % 32 == 0 && GLOAD_WARPS <= GEXP_WARPS, "expander warps");
constexpr long long WAIT_CYCLES = 2000000000ll;  // ~1 s at 2 GHz before giving up
// The 0/1 operands are 0 and e4m3 0x08 = 2^-6 (a normal number): products
// are 0 or 2^-12 and a count c accumulates to c * 2^-12, exact in fp32 for
// c < 2^24; the epilogue scales back by 2^12.
constexpr float GRAM_UNIT_INV = 4096.0f;

// Byte offset of element (rank r, K position k) inside a tile of GK-row
// chunks: core matrix (r/8, k/16) at (r/8)*GSBO + (k/16)*128, element
// (r%8)*16 + k%16.
__device__ __forceinline__ uint32_t core_offset(uint32_t r, uint32_t k) {
  return (r >> 3) * GSBO + (k >> 4) * 128u + (r & 7u) * 16u + (k & 15u);
}

// Rows j, j + 8, j + 16 and j + 24 of a 32-row column word x as four e4m3
// bytes of 0 or 0x08: bit j + 8q moves to bit 8q + 3 with one shift, and the
// mask keeps those bits. A chunk's rows are thus laid out along K in a fixed
// order that is not row order; A and B use the same order, so every product
// X[a][t] * X[b][t] is still formed once and the contraction over the chunk's
// rows is unchanged.
template <uint32_t J>
__device__ __forceinline__ uint32_t spread_rows(uint32_t x) {
  return (J <= 3 ? (x << (3 - J)) : (x >> (J - 3))) & 0x08080808u;
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
constexpr uint32_t GRAM_IDESC = (1u << 4) | ((GN >> 3) << 17) | ((GM >> 4) << 24);

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
// Tile pairs: A tile i (ranks 128 i ..) with every B tile J (ranks 256 J ..)
// that holds a rank above one of A's, i.e. J >= i / 2.
__host__ __device__ __forceinline__ uint32_t gram_pairs_of(uint32_t na, uint32_t nb) {
  uint32_t p = 0;
  for (uint32_t i = 0; i < na; ++i) p += nb > i / 2 ? nb - i / 2 : 0u;
  return p;
}

// ALL = false: the pair cohort's counts over stop g's block are added to its
// counters (atomics; `nsplit` CTAs split each tile pair's rows).
// ALL = true: CTA (block b, tile pair) writes the pairs' counts over block b
// of the pass to pc[b * pairs + record] (plain stores; every pair of frequent
// ranks gets one, zeros included), for all blocks in one launch; with
// `nsplit` > 1 (32-bit counts) nsplit CTAs split the block's rows and add
// their partial counts to the zeroed array.
template <bool ALL, class T>
__global__ void __launch_bounds__(GRAM_THREADS, 1) k_gram_pairs(Lattice L, uint32_t nsplit,
                                                                uint32_t kre, T *pc) {
  extern __shared__ __align__(1024) uint8_t gsm[];
  __shared__ __align__(8) uint64_t full[GSTAGES], empty[GSTAGES], done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile uint32_t failed;
  Ctrl *C = L.ctrl;
  if (!ALL) {
    pdl_wait();
    pdl_trigger();
    if (!gram_may_run(L, C, kre)) return;
  }
  const uint32_t na = (L.l1 + GM - 1) / GM, nb = (L.l1 + GN - 1) / GN;
  const uint32_t ntp = gram_pairs_of(na, nb);
  // stop g whose block this CTA counts (ALL: the stop of pass block b)
  const uint32_t g = ALL ? blockIdx.x / (ntp * nsplit) + 1 : C->step;
  uint32_t stop;
  uint64_t first, last;
  block_of(g, L.stop_max, L.M, L.n, &stop, &first, &last);
  const uint32_t nrows = (uint32_t)(last - first);
  if (!ALL && blockIdx.x == 0 && threadIdx.x == 0) C->gram_rows += nrows;
  const uint32_t nkc = (nrows + GK - 1) / GK;
  // which tile pair (A tile ti, B tile tj >= ti / 2) and which K split
  const uint32_t pair = ALL ? (blockIdx.x / nsplit) % ntp : blockIdx.x / nsplit;
  const uint32_t split = blockIdx.x % nsplit;
  uint32_t ti = 0, rem = pair;
  while (ti < na && rem >= nb - ti / 2) { rem -= nb - ti / 2; ++ti; }
  if (ti >= na) return;
  const uint32_t tj = ti / 2 + rem;
  const uint32_t per = (nkc + nsplit - 1) / nsplit;
  const uint32_t kc0 = split * per;
  const uint32_t kc1 = kc0 + per < nkc ? kc0 + per : nkc;
  if (kc0 >= kc1) return;  // nothing to count for this split (uniform per CTA)
  const uint32_t nk = kc1 - kc0;
  uint8_t *stage_a = gsm;                      // GSTAGES x 16 KiB
  uint8_t *stage_b = gsm + GSTAGES * GTILE_A;  // GSTAGES x 32 KiB
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (uint32_t s = 0; s < GSTAGES; ++s) {
      mbar_init(&full[s], GLOAD_WARPS);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    failed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == GEXP_WARPS) {  // tensor memory: 256 columns of 128 lanes (fp32)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;"
                 ::"r"(sm_addr(&tmem_base)) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;

  if (warp < GLOAD_WARPS) {
    // expanders: thread rr owns rank row rr (the A tile's 128, then the B
    // tile's 256) and writes its GK rows of every chunk; the rank's eight
    // column words of a chunk are two 16-byte loads, issued GPREFETCH chunks
    // ahead
    const uint32_t rr = threadIdx.x;
    const bool is_a = rr < GM;
    const uint64_t rank = is_a ? (uint64_t)ti * GM + rr : (uint64_t)tj * GN + (rr - GM);
    const bool ok = rank < L.l1;
    const uint32_t tw = L.tw, st = bs_stride((int)tw);
    const uint32_t tw_shift = __ffs(tw) - 1;  // tw is 4, 8 or 16: a chunk's 4 words share a tile
    const uint64_t tile_words = (uint64_t)L.l1p * st;
    const uint32_t *col = vcols(L, g) + (ok ? rank : 0) * st;
    uint8_t *row0 = gsm + (is_a ? 0u : GSTAGES * GTILE_A) + core_offset(is_a ? rr : rr - GM, 0);
    const uint32_t stage_bytes = is_a ? GTILE_A : GTILE_B;
    // the block's words end at a whole tile; a chunk's words past them
    // (4-word tiles: the last chunk may reach past the last tile) read as 0
    const uint32_t nw32 = (nrows + 31) / 32, wpad = (nw32 + tw - 1) / tw * tw;
    auto load = [&](uint32_t kc, uint32_t h) -> uint4 {
      const uint32_t w0 = kc * (GK / 32) + 4 * h;
      return ok && w0 < wpad
                 ? __ldg(reinterpret_cast<const uint4 *>(col + (w0 >> tw_shift) * tile_words +
                                                         (w0 & (tw - 1))))
                 : make_uint4(0u, 0u, 0u, 0u);
    };
    uint4 q[GPREFETCH][GQ];
#pragma unroll
    for (uint32_t d = 0; d < GPREFETCH; ++d)
#pragma unroll
      for (uint32_t h = 0; h < GQ; ++h)
        q[d][h] = d < nk ? load(kc0 + d, h) : make_uint4(0, 0, 0, 0);
    for (uint32_t i0 = 0; i0 < nk; i0 += GPREFETCH) {
#pragma unroll
      for (uint32_t d = 0; d < GPREFETCH; ++d) {
        const uint32_t i = i0 + d;
        if (i >= nk || __shfl_sync(0xffffffffu, failed, 0)) break;  // warp-uniform
        const uint32_t s = i % GSTAGES, use = i / GSTAGES;
        uint4 w[GQ];
#pragma unroll
        for (uint32_t h = 0; h < GQ; ++h) {
          w[h] = q[d][h];
          if (i + GPREFETCH < nk) q[d][h] = load(kc0 + i + GPREFETCH, h);
        }
        // one lane per warp waits for the ring slot and one arrives for the
        // warp (the barrier counts warps, not threads)
        bool slot_ok = true;
        if (use > 0 && lane == 0) slot_ok = mbar_wait(&empty[s], (use - 1) & 1);
        if (!__shfl_sync(0xffffffffu, slot_ok ? 1u : 0u, 0)) { failed = 1; break; }
        uint8_t *dst = row0 + s * stage_bytes;
        // core matrix columns 2v and 2v + 1 take word v's 32 rows: bytes of
        // rows {j, j+8, j+16, j+24} for j = 0..3, then for j = 4..7
#pragma unroll
        for (uint32_t v = 0; v < 4 * GQ; ++v) {
          const uint4 &wq = w[v / 4];
          const uint32_t x = v % 4 == 0 ? wq.x : v % 4 == 1 ? wq.y : v % 4 == 2 ? wq.z : wq.w;
          *reinterpret_cast<uint4 *>(dst + (2 * v) * 128u) =
              make_uint4(spread_rows<0>(x), spread_rows<1>(x), spread_rows<2>(x),
                         spread_rows<3>(x));
          *reinterpret_cast<uint4 *>(dst + (2 * v + 1) * 128u) =
              make_uint4(spread_rows<4>(x), spread_rows<5>(x), spread_rows<6>(x),
                         spread_rows<7>(x));
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[s]);
      }
    }
  } else if (warp == GEXP_WARPS && lane == 0) {
    // MMA issuer: 8 instructions (K = 32 bytes each) per 256-row chunk
    for (uint32_t i = 0; i < nk; ++i) {
      const uint32_t s = i % GSTAGES, use = i / GSTAGES;
      if (failed || !mbar_wait(&full[s], use & 1)) { failed = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = sm_addr(stage_a + s * GTILE_A);
      const uint32_t b0 = sm_addr(stage_b + s * GTILE_B);
#pragma unroll
      for (uint32_t k = 0; k < GK / 32; ++k)
        mma_f8(tmem, smem_desc(a0 + k * 256, 128, GSBO), smem_desc(b0 + k * 256, 128, GSBO),
               (i | k) != 0);
      mma_commit(&empty[s]);
    }
    mma_commit(&done);  // arrives once every MMA issued above has completed
  }
  __syncwarp();
  // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (ranks of A tile
  // ti), columns 64 (w / 4) .. +63 (ranks of B tile tj)
  if (lane == 0 && !mbar_wait(&done, 0)) failed = 1;
  __syncthreads();
  const bool ok = !failed;  // the same for every thread of the CTA
  if (threadIdx.x == 0 && !ok) C->error = 5;  // DIC_ETIMEOUT
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok && warp < GEXP_WARPS) {
    // Each warp stages 32 x 32 sub-tiles through shared memory (the operand
    // rings are idle once `done` has fired) so that a warp's adds go to 32
    // consecutive counters: lane q adds count (a, b0 + q) of row a.
    const uint64_t l1 = L.l1;
    T *pc_out = ALL ? pc + (uint64_t)(g - 1) * (l1 * (l1 - 1) / 2) : pc;
    uint32_t *stage = reinterpret_cast<uint32_t *>(gsm) + warp * (32 * 33);
    const uint32_t lq = warp % 4;
    const uint64_t a0 = (uint64_t)ti * GM + lq * 32;
    for (uint32_t c0 = (warp / 4) * 64; c0 < (warp / 4) * 64 + 64; c0 += 32) {
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
      const uint64_t b = (uint64_t)tj * GN + c0 + lane;
      if (a0 >= l1 || (uint64_t)tj * GN + c0 + 31 <= a0) continue;  // all b <= a (warp-uniform)
#pragma unroll
      for (int k = 0; k < 32; ++k)
        stage[lane * 33 + k] = (uint32_t)(__uint_as_float(v[k]) * GRAM_UNIT_INV);
      __syncwarp();
      const uint32_t rmax = l1 - a0 < 32 ? (uint32_t)(l1 - a0) : 32u;
      for (uint32_t r = 0; r < rmax; ++r) {
        const uint64_t a = a0 + r;
        const uint32_t cnt = stage[r * 33 + lane];
        if (ALL) {
          if (b > a && b < l1) {
            if (nsplit == 1) {
              pc_out[pair_record(a, b, l1)] = (T)cnt;
            } else if (cnt) {  // K splits (32-bit counts only) meet in L2
              if constexpr (sizeof(T) == 4) atomicAdd(&pc_out[pair_record(a, b, l1)], cnt);
            }
          }
        } else if (b > a && b < l1 && cnt) {
          atomicAdd(&L.csupp[pair_record(a, b, l1)], cnt);
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == GEXP_WARPS)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// -------------------------------------------------------------- launchers
uint32_t gram_tile_pairs(uint32_t l1) {
  return gram_pairs_of((l1 + GM - 1) / GM, (l1 + GN - 1) / GN);
}
uint32_t gram_chunks(uint64_t rows) { return (uint32_t)((rows + GK - 1) / GK); }

cudaError_t launch_gram_pairs(Lattice L, uint32_t nsplit, uint32_t kre, cudaStream_t s) {
  const uint32_t npairs = gram_tile_pairs(L.l1);
  const size_t smem = GSTAGES * (GTILE_A + GTILE_B);  // the A and B rings
  auto kern = k_gram_pairs<false, uint32_t>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<npairs * nsplit, GRAM_THREADS, smem, s>>>(L, nsplit, kre, (uint32_t *)nullptr);
  return cudaGetLastError();
}

// A pass of few large blocks gives fewer (block, tile pair) CTAs than SMs:
// with 32-bit counts each block's rows are then split across nsplit CTAs
// (at least 16 chunks each) whose partial counts are added into the zeroed
// count array.
template <class T>
static cudaError_t gram_all(Lattice L, T *pc, cudaStream_t s) {
  const uint64_t grid = (uint64_t)gram_tile_pairs(L.l1) * L.stop_max;
  if (grid == 0 || grid > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t nsplit = 1;
  if (sizeof(T) == 4 && grid < (uint64_t)sms) {
    const uint64_t blockmax = L.M < L.n ? L.M : L.n;
    const uint64_t by_chunks = gram_chunks(blockmax) / 16;
    const uint64_t want = ((uint64_t)sms + grid - 1) / grid;
    nsplit = (uint32_t)std::max<uint64_t>(1, std::min(want, by_chunks));
  }
  if (nsplit > 1) {
    const uint64_t l1 = L.l1;
    cudaError_t e = cudaMemsetAsync(pc, 0, (size_t)L.stop_max * (l1 * (l1 - 1) / 2) * sizeof(T), s);
    if (e != cudaSuccess) return e;
  }
  const size_t smem = GSTAGES * (GTILE_A + GTILE_B);
  auto kern = k_gram_pairs<true, T>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)(grid * nsplit), GRAM_THREADS, smem, s>>>(L, nsplit, 0u, pc);
  return cudaGetLastError();
}

cudaError_t launch_gram_all_blocks(Lattice L, void *pc, bool wide, cudaStream_t s) {
  if (!L.vall) return cudaErrorInvalidValue;
  return wide ? gram_all<uint32_t>(L, (uint32_t *)pc, s) : gram_all<uint16_t>(L, (uint16_t *)pc, s);
}

// ---------------------------------------------------------- pair events
// Algorithm 4 for the pair cohort over its whole pass, from the per-block
// counts pc[b][record] of the all-blocks GEMM: pair c (born before stop 1) is
// promoted at the first stop g with support >= minsup, or dropped at the
// first stop where its bound support + M * (stop_max - g) is below minsup
// (exactly one of the two happens by stop_max). Its counter receives the
// full-pass total; ev[c] = 2g + 1 (promoted at g) or 2g (dropped at g);
// hist[g] / hist[stop_max + 2 + g] count promotions / drops per stop.
template <class T>
__global__ void __launch_bounds__(256) k_pair_events(Lattice L, const T *__restrict__ pc,
                                                     uint32_t *ev, uint32_t *hist) {
  extern __shared__ uint32_t sh[];
  const uint32_t S = L.stop_max, H = 2 * (S + 2);
  const bool local = H <= 4096;
  if (local) {
    for (uint32_t i = threadIdx.x; i < H; i += blockDim.x) sh[i] = 0;
    __syncthreads();
  }
  const uint64_t np = (uint64_t)L.l1 * (L.l1 - 1) / 2;
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < np) {
    uint64_t cum = 0;
    uint32_t e = 0;
    for (uint32_t g = 1; g <= S; ++g) {
      cum += pc[(uint64_t)(g - 1) * np + c];
      if (e) continue;
      if (cum >= L.minsup) e = 2 * g + 1;
      else if (cum + L.M * (uint64_t)(S - g) < (uint64_t)L.minsup) e = 2 * g;
    }
    L.csupp[c] = (uint32_t)cum;
    ev[c] = e;
    const uint32_t slot = (e & 1u) ? (e >> 1) : S + 2 + (e >> 1);
    if (local) atomicAdd(&sh[slot], 1u);
    else atomicAdd(&hist[slot], 1u);
  }
  if (local) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < H; i += blockDim.x)
      if (sh[i]) atomicAdd(&hist[i], sh[i]);
  }
}

// One CTA: ev_off[g] = promotions before stop g (exclusive scan over stops
// 1..stop_max, ev_off[stop_max + 1] = all of them), a cursor copy for the
// scatter, ev_pruned[g] = drops at g, ev_pruned[0] = all promotions.
__global__ void __launch_bounds__(1024) k_pair_events_scan(Lattice L, const uint32_t *hist,
                                                           uint32_t *ev_off, uint32_t *cursor,
                                                           uint32_t *ev_pruned) {
  __shared__ uint32_t part[1024];
  const uint32_t S = L.stop_max;
  const uint32_t per = (S + 1023) / 1024;
  const uint32_t g0 = 1 + threadIdx.x * per;
  uint32_t sum = 0;
  for (uint32_t g = g0; g < g0 + per && g <= S; ++g) sum += hist[g];
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int i = 0; i < 1024; ++i) { const uint32_t v = part[i]; part[i] = run; run += v; }
    ev_off[0] = 0;
    ev_off[S + 1] = run;
    ev_pruned[0] = run;
  }
  __syncthreads();
  uint32_t run = part[threadIdx.x];
  for (uint32_t g = g0; g < g0 + per && g <= S; ++g) {
    ev_off[g] = run;
    cursor[g] = run;
    ev_pruned[g] = hist[S + 2 + g];
    run += hist[g];
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // stop 1's range, read by its count kernel
    Ctrl *C = L.ctrl;
    C->ev_next[3] = ev_off[1];
    C->ev_next[4] = ev_off[2];
    C->ev_next[5] = ev_pruned[1];
    C->ev_stop[1] = 1;
  }
}

// The promoted pairs grouped by promotion stop (order within a stop is
// irrelevant: MAKECANDIDATES depends only on the set).
__global__ void __launch_bounds__(256) k_pair_events_scatter(Lattice L, const uint32_t *ev,
                                                             uint32_t *cursor, uint32_t *ev_list) {
  const uint64_t np = (uint64_t)L.l1 * (L.l1 - 1) / 2;
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= np) return;
  const uint32_t e = ev[c];
  if (e & 1u) ev_list[atomicAdd(&cursor[e >> 1], 1u)] = (uint32_t)c;
}

cudaError_t launch_pair_events(Lattice L, const void *pc, bool wide, uint32_t *ev,
                               uint32_t *hist, uint32_t *ev_off, uint32_t *cursor,
                               uint32_t *ev_list, uint32_t *ev_pruned, cudaStream_t s) {
  const uint64_t np = (uint64_t)L.l1 * (L.l1 - 1) / 2;
  if (np == 0) return cudaSuccess;
  const uint64_t grid = (np + 255) / 256;
  if (grid > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  const uint32_t H = 2 * (L.stop_max + 2);
  const size_t smem = H <= 4096 ? (size_t)H * 4 : 0;
  cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)H * 4, s);
  if (e != cudaSuccess) return e;
  if (wide)
    k_pair_events<uint32_t><<<(unsigned)grid, 256, smem, s>>>(L, (const uint32_t *)pc, ev, hist);
  else
    k_pair_events<uint16_t><<<(unsigned)grid, 256, smem, s>>>(L, (const uint16_t *)pc, ev, hist);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_pair_events_scan<<<1, 1024, 0, s>>>(L, hist, ev_off, cursor, ev_pruned);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_pair_events_scatter<<<(unsigned)grid, 256, 0, s>>>(L, ev, cursor, ev_list);
  return cudaGetLastError();
}

}  // namespace dic
