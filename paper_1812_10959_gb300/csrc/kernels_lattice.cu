// Device lattice of ParallelDIC (Algorithm 2) on sm_103a: the first pass,
// the bitmap packer, column compaction, the pair join, PRUNE (Algorithm 4),
// the box set, MAKECANDIDATES and CHECKFULLPASS (Algorithm 5).
//
// Layout: candidate records live in one append-only array. Records created
// at the same stop form a contiguous cohort; since every record is counted
// once per stop from its creation on, a cohort completes its full pass (and
// leaves DASHED for SOLID, Algorithm 5) all at once, so DASHED is the window
// [head, tail) and solidifying is advancing `head` past whole cohorts. PRUNE
// erases records in place (shape NIL); the count kernels skip them.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"
#include "lattice_device.cuh"

namespace dic {

// --------------------------------------------------------- first pass
// supp1[i] = number of rows with bit i set, over all n rows (FIRSTPASS of
// Section 4.2). Each thread owns one 64-bit word column j and a strided set
// of rows and keeps a bit-sliced counter of the column: plane k holds bit k
// of the 64 items' counts. Words are added sixteen at a time through a
// carry-save adder tree (Harley-Seal: a full adder per bit position is one
// XOR3 and one majority, a LOP3 each per 32-bit half), so a word costs about
// eight integer instructions instead of a transposition. At the end the
// threads of a column add their counters with bit-sliced ripple adders in
// shared memory, and a warp turns each column's planes into 64 counts (lane b
// reads bit b of every plane) with one atomic per item per CTA.
constexpr uint32_t IC_THREADS = 256;
constexpr int IC_PLANES = 21;  // counts below 2^21 per CTA (the launch keeps them there)

// One full-adder column step: sum and carry of a + b + c, bitwise.
__device__ __forceinline__ void csa(uint64_t &h, uint64_t &l, uint64_t a, uint64_t b,
                                    uint64_t c) {
  const uint64_t u = a ^ b;
  h = (a & b) | (u & c);
  l = u ^ c;
}

// Add sixteen words to the bit-sliced counter P (planes 0-3 take the tree's
// ones, twos, fours and eights; its sixteens ripple into planes 4 and up).
__device__ __forceinline__ void csa16(uint64_t (&P)[IC_PLANES], const uint64_t (&x)[16]) {
  uint64_t twosA, twosB, foursA, foursB, eightsA, eightsB, sixteens;
  csa(twosA, P[0], P[0], x[0], x[1]);
  csa(twosB, P[0], P[0], x[2], x[3]);
  csa(foursA, P[1], P[1], twosA, twosB);
  csa(twosA, P[0], P[0], x[4], x[5]);
  csa(twosB, P[0], P[0], x[6], x[7]);
  csa(foursB, P[1], P[1], twosA, twosB);
  csa(eightsA, P[2], P[2], foursA, foursB);
  csa(twosA, P[0], P[0], x[8], x[9]);
  csa(twosB, P[0], P[0], x[10], x[11]);
  csa(foursA, P[1], P[1], twosA, twosB);
  csa(twosA, P[0], P[0], x[12], x[13]);
  csa(twosB, P[0], P[0], x[14], x[15]);
  csa(foursB, P[1], P[1], twosA, twosB);
  csa(eightsB, P[2], P[2], foursA, foursB);
  csa(sixteens, P[3], P[3], eightsA, eightsB);
  uint64_t carry = sixteens;
#pragma unroll
  for (int k = 4; k < IC_PLANES; ++k) {
    const uint64_t t = P[k] & carry;
    P[k] ^= carry;
    carry = t;
  }
}

// Columns of JC words per CTA (blockIdx.y picks the chunk), IC_THREADS / JC
// row threads per column; JC = 32, or the power of two at least W below 32,
// so a warp's loads cover consecutive words of consecutive rows.
template <uint32_t JC>
__global__ void __launch_bounds__(IC_THREADS) k_item_count(const uint64_t *__restrict__ B,
                                                           uint64_t n, uint32_t W, uint32_t m,
                                                           uint32_t *__restrict__ cnt) {
  constexpr uint32_t RT = IC_THREADS / JC;
  __shared__ uint64_t sp[IC_PLANES][IC_THREADS];
  const uint32_t t = threadIdx.x, jl = t % JC, rt = t / JC;
  const uint32_t j = blockIdx.y * JC + jl;
  const bool col = j < W;
  const uint64_t stride = (uint64_t)gridDim.x * RT;
  uint64_t P[IC_PLANES];
#pragma unroll
  for (int k = 0; k < IC_PLANES; ++k) P[k] = 0;
  uint64_t r = (uint64_t)blockIdx.x * RT + rt;
  for (; r + 15 * stride < n; r += 16 * stride) {
    uint64_t x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = col ? __ldcs(B + (r + i * stride) * W + j) : 0ull;
    csa16(P, x);
  }
  if (r < n) {  // the last rows of this thread (fewer than sixteen)
    uint64_t x[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const uint64_t rr = r + i * stride;
      x[i] = (col && rr < n) ? __ldcs(B + rr * W + j) : 0ull;
    }
    csa16(P, x);
  }
  // the row threads of a column add their counters: at each step the upper
  // half hands its planes over through shared memory (ripple-carry adders,
  // bitwise; the totals fit the planes)
  for (uint32_t step = RT / 2; step >= 1; step >>= 1) {
    if (rt >= step && rt < 2 * step)
#pragma unroll
      for (int k = 0; k < IC_PLANES; ++k) sp[k][t] = P[k];
    __syncthreads();
    if (rt < step) {
      uint64_t c = 0;
#pragma unroll
      for (int k = 0; k < IC_PLANES; ++k) {
        const uint64_t b = sp[k][t + step * JC];
        uint64_t h, l;
        csa(h, l, P[k], b, c);
        P[k] = l;
        c = h;
      }
    }
    __syncthreads();
  }
  if (rt == 0)
#pragma unroll
    for (int k = 0; k < IC_PLANES; ++k) sp[k][jl] = P[k];
  __syncthreads();
  // a warp per column: lane b gathers bit b (and b + 32) of every plane
  const uint32_t lane = t & 31, warp = t >> 5;
  for (uint32_t c = warp; c < JC; c += IC_THREADS / 32) {
    const uint32_t jc = blockIdx.y * JC + c;
    if (jc >= W) continue;
    uint32_t v0 = 0, v1 = 0;
#pragma unroll
    for (int k = 0; k < IC_PLANES; ++k) {
      const uint64_t pk = sp[k][c];
      v0 |= (uint32_t)((pk >> lane) & 1u) << k;
      v1 |= (uint32_t)((pk >> (lane + 32)) & 1u) << k;
    }
    const uint32_t i0 = jc * 64 + lane, i1 = i0 + 32;
    if (i0 < m && v0) atomicAdd(&cnt[i0], v0);
    if (i1 < m && v1) atomicAdd(&cnt[i1], v1);
  }
}

template <uint32_t JC>
static cudaError_t go_item_count(const uint64_t *B, uint64_t n, uint32_t W, uint32_t m,
                                 uint32_t *cnt, int sms, cudaStream_t s) {
  constexpr uint32_t RT = IC_THREADS / JC;
  // two CTAs per SM over the column chunks, and enough CTAs that the rows one
  // CTA adds up (its column totals) stay below 2^IC_PLANES
  const uint32_t ny = (W + JC - 1) / JC;
  uint64_t gx = std::max<uint64_t>(1, (uint64_t)sms * 2 / ny);
  const uint64_t cap = ((uint64_t)1 << IC_PLANES) - 1;
  gx = std::max<uint64_t>(gx, (n + cap - 1) / cap);
  gx = std::min<uint64_t>(gx, std::max<uint64_t>(1, (n + RT - 1) / RT));
  if (gx > 0x7FFFFFFFull || ny > 65535) return cudaErrorInvalidValue;
  k_item_count<JC><<<dim3((unsigned)gx, ny), IC_THREADS, 0, s>>>(B, n, W, m, cnt);
  return cudaGetLastError();
}

cudaError_t launch_item_count(const uint64_t *B, uint64_t n, uint32_t W, uint32_t m,
                              uint32_t *cnt, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)m * 4, s);
  if (e != cudaSuccess || n == 0) return e;
  if (W >= 32) return go_item_count<32>(B, n, W, m, cnt, sms, s);
  if (W > 8) return go_item_count<16>(B, n, W, m, cnt, sms, s);
  if (W > 4) return go_item_count<8>(B, n, W, m, cnt, sms, s);
  if (W > 2) return go_item_count<4>(B, n, W, m, cnt, sms, s);
  if (W > 1) return go_item_count<2>(B, n, W, m, cnt, sms, s);
  return go_item_count<1>(B, n, W, m, cnt, sms, s);
}

// ----------------------------------------------------- column compaction
// Bc[t] keeps only the frequent items of B[t], renumbered by rank (rank
// order = item order). Exact: a candidate never contains an infrequent item
// (Section 4.2: infrequent 1-itemsets and their supersets are pruned).
// One warp per row; the output row is assembled in shared memory.
__global__ void __launch_bounds__(256) k_compact_rows(const uint64_t *__restrict__ B, uint64_t n,
                                                      uint32_t W,
                                                      const int32_t *__restrict__ rank_of,
                                                      uint64_t *__restrict__ Bc, uint32_t wc) {
  extern __shared__ unsigned long long sbuf[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long *out = sbuf + (size_t)warp * wc;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  for (uint64_t row = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp; row < n; row += nwarps) {
    for (uint32_t j = lane; j < wc; j += 32) out[j] = 0ull;
    __syncwarp();
    for (uint32_t j = lane; j < W; j += 32) {
      uint64_t x = __ldcs(B + row * W + j);
      while (x) {
        const uint32_t b = (uint32_t)(__ffsll((long long)x) - 1);
        x &= x - 1;
        const int32_t r = __ldg(rank_of + j * 64 + b);
        if (r >= 0) atomicOr(&out[r >> 6], 1ull << (r & 63));
      }
    }
    __syncwarp();
    for (uint32_t j = lane; j < wc; j += 32) Bc[row * wc + j] = out[j];
    __syncwarp();
  }
}

cudaError_t launch_compact_rows(const uint64_t *B, uint64_t n, uint32_t W, const int32_t *rank_of,
                                uint64_t *Bc, uint32_t wc, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = (size_t)8 * wc * 8;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_compact_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  uint64_t want = (n + 7) / 8;
  int grid = (int)(want < (uint64_t)sms * 8 ? want : (uint64_t)sms * 8);
  k_compact_rows<<<grid, 256, smem, s>>>(B, n, W, rank_of, Bc, wc);
  return cudaGetLastError();
}

// ------------------------------------------------------------ packing
// BitMask of Section 4.1 from CSR item lists: bit p%64 of word p/64.
__global__ void k_pack_csr(const uint64_t *__restrict__ row_ptr, const uint32_t *__restrict__ items,
                           uint64_t n, uint32_t m, uint32_t W, unsigned long long *words,
                           uint32_t *bad) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const uint64_t b = row_ptr[t], e = row_ptr[t + 1];
    for (uint64_t j = b; j < e; ++j) {
      const uint32_t it = items[j];
      if (it >= m) { atomicOr(bad, 1u); continue; }
      atomicOr(&words[t * W + (it >> 6)], 1ull << (it & 63));
    }
  }
}

cudaError_t launch_pack_csr(const uint64_t *row_ptr, const uint32_t *items, uint64_t n, uint32_t m,
                            uint32_t W, uint64_t *words, uint32_t *bad, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  uint64_t want = (n + 255) / 256;
  int grid = (int)(want < 65535ull * 4 ? want : 65535ull * 4);
  k_pack_csr<<<grid, 256, 0, s>>>(row_ptr, items, n, m, W, (unsigned long long *)words, bad);
  return cudaGetLastError();
}

// Every bit at an item position >= m must be zero.
__global__ void k_check_padding(const uint64_t *__restrict__ words, uint64_t n, uint32_t m,
                                uint32_t W, uint32_t *bad) {
  const uint32_t used = m - (W - 1) * 64;  // items in the last word, 1..64
  const uint64_t pad = used == 64 ? 0ull : ~((1ull << used) - 1);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
    if (words[t * W + W - 1] & pad) atomicOr(bad, 1u);
}

cudaError_t launch_check_padding(const uint64_t *words, uint64_t n, uint32_t m, uint32_t W,
                                 uint32_t *bad, cudaStream_t s) {
  if (n == 0 || m % 64 == 0) return cudaSuccess;
  uint64_t want = (n + 255) / 256;
  int grid = (int)(want < 65535ull * 4 ? want : 65535ull * 4);
  k_check_padding<<<grid, 256, 0, s>>>(words, n, m, W, bad);
  return cudaGetLastError();
}

// ------------------------------------------------------------ pair join
// DASHED <- every pair {a,b}, a<b, of frequent items as circles (the
// bitwise-OR join of the first pass, Section 4.2), in lexicographic order.
__device__ __forceinline__ uint64_t pair_off(uint64_t a, uint64_t l1) {
  return a * (2 * l1 - a - 1) / 2;  // pairs whose first rank is < a
}

// CTA per first rank a: the records of pairs {a, b}, b = a+1 .. l1-1, are
// the contiguous range pair_off(a) + (b - a - 1), so their mask words and
// fields are written with consecutive addresses.
__global__ void __launch_bounds__(256) k_pair_join(Lattice L) {
  const uint64_t l1 = L.l1;
  const uint32_t wc = L.wc;
  for (uint64_t a = blockIdx.x; a + 1 < l1; a += gridDim.x) {
    const uint64_t p0 = pair_off(a, l1), cnt = l1 - a - 1;
    uint64_t *mk = L.cmask + p0 * wc;
    for (uint64_t e = threadIdx.x; e < cnt * wc; e += blockDim.x) {
      const uint64_t b = a + 1 + e / wc;
      const uint32_t w = (uint32_t)(e % wc);
      uint64_t word = 0;
      if ((a >> 6) == w) word |= 1ull << (a & 63);
      if ((b >> 6) == w) word |= 1ull << (b & 63);
      mk[e] = word;
    }
    for (uint64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
      const uint64_t p = p0 + q, b = a + 1 + q;
      L.csupp[p] = 0;
      L.cbirth[p] = 0;
      L.cshape[p] = SH_CIRCLE;
      L.cpromo[p] = ~0u;
      L.ck[p] = 2;
      uint4 *rk = reinterpret_cast<uint4 *>(L.cranks + p * KRMAX);
      rk[0] = make_uint4((uint32_t)a | ((uint32_t)b << 16), 0u, 0u, 0u);
      rk[1] = make_uint4(0u, 0u, 0u, 0u);
    }
  }
}

// Algorithm 1's start: Dashed Circle holds every 1-itemset (rank r is record
// r); with no first pass the ranks are all m items.
__global__ void k_singleton_join(Lattice L) {
  const uint64_t total = (uint64_t)L.l1 * L.wc;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t r = (uint32_t)(i / L.wc), w = (uint32_t)(i % L.wc);
    L.cmask[i] = (r >> 6) == w ? 1ull << (r & 63) : 0ull;
    if (w == 0) {
      L.csupp[r] = 0;
      L.cbirth[r] = 0;
      L.cshape[r] = SH_CIRCLE;
      L.cpromo[r] = ~0u;
      L.ck[r] = 1;
      L.cranks[(uint64_t)r * KRMAX] = (uint16_t)r;
    }
  }
}

cudaError_t launch_singleton_join(Lattice L, cudaStream_t s) {
  const uint64_t total = (uint64_t)L.l1 * L.wc;
  const uint64_t want = (total + 255) / 256;
  const int grid = (int)(want < 65535ull * 4 ? (want ? want : 1) : 65535ull * 4);
  k_singleton_join<<<grid, 256, 0, s>>>(L);
  return cudaGetLastError();
}

cudaError_t launch_pair_join(Lattice L, uint64_t npairs, cudaStream_t s) {
  if (npairs == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t rows = (uint64_t)L.l1 - 1;
  const int grid = (int)(rows < (uint64_t)sms * 8 ? rows : (uint64_t)sms * 8);
  k_pair_join<<<grid, 256, 0, s>>>(L);
  return cudaGetLastError();
}

// --------------------------------------------------------------- PRUNE
// Algorithm 4 over the dashed records after the count of stop g (the ROWS
// path; the fast count paths apply the same rule in their epilogue). The
// superset loop of Algorithm 4 is not run: every (k-1)-subset of a record is
// a box when it is generated and boxes never change shape, so a dashed
// circle has no dashed superset and the loop could only match the record
// itself.
__global__ void __launch_bounds__(256) k_promote(Lattice L) {
  pdl_wait();
  pdl_trigger();
  Ctrl *C = L.ctrl;
  if (C->stall || C->done) return;
  const uint32_t g = C->step, tail = C->tail;
  const uint32_t head = counted_lo(L, C->head, tail, g, false);
  uint32_t pruned = 0, solid = 0;
  apply_pair_events(L, C, g, (uint64_t)blockIdx.x * blockDim.x + threadIdx.x,
                    (uint64_t)gridDim.x * blockDim.x, pruned, solid);
  for (uint32_t c = head + blockIdx.x * blockDim.x + threadIdx.x; c < tail;
       c += gridDim.x * blockDim.x)
    settle_record(L, C, c, L.csupp[c], g, false, pruned, solid);
  block_add_tallies(C, pruned, solid, 0ull);
}

cudaError_t launch_promote(Lattice L, int grid, cudaStream_t s) {
  return launch_k(k_promote, grid, 256, 0, s, L);
}

// -------------------------------------------------------------- box set
// Insert the records promoted at this stop (ROWS path). The load check runs
// before any insert and reads only values this kernel does not change, so
// every block takes the same decision.
__global__ void __launch_bounds__(256) k_hash_insert(Lattice L) {
  pdl_wait();
  pdl_trigger();
  Ctrl *C = L.ctrl;
  if (C->stall || C->done) return;
  const uint32_t P = C->n_newbox;
  if ((uint64_t)(C->hash_used + P) * 2 > L.hcap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) C->stall = ST_HASH;
    return;
  }
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const uint32_t c = L.newbox[p];
    const uint64_t sum = mask_hash_sum(L.cmask + (uint64_t)c * L.wc, L.wc);
    L.newhash[p] = sum;
    box_insert(L, c, sum);
  }
}

cudaError_t launch_hash_insert(Lattice L, int grid, cudaStream_t s) {
  return launch_k(k_hash_insert, grid, 256, 0, s, L);
}

// Rebuild the box set into a larger table.
__global__ void k_rehash(Lattice L, const uint32_t *oslot, uint32_t ocap) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < ocap; s += gridDim.x * blockDim.x) {
    const uint32_t v = oslot[s];
    if (!v) continue;
    box_insert(L, v - 1, mask_hash_sum(L.cmask + (uint64_t)(v - 1) * L.wc, L.wc));
  }
}

cudaError_t launch_rehash(Lattice L, const uint32_t *oslot, uint32_t ocap, cudaStream_t s) {
  if (ocap == 0) return cudaSuccess;
  int grid = (int)((ocap + 255) / 256 < 65535u * 4 ? (ocap + 255) / 256 : 65535u * 4);
  k_rehash<<<grid, 256, 0, s>>>(L, oslot, ocap);
  return cudaGetLastError();
}

// ------------------------------------------------------ MAKECANDIDATES
// New candidates at stop g: C = A u {r} for a record A promoted at g and a
// rank r not in A, kept iff every |C|-1 subset C \ {j} is a box. Each such
// C has one or more promoted-at-g parents C \ {j}; only the parent with the
// smallest j emits it, so every C appears exactly once without a dedup
// table: thread (A, r) emits iff no j < r in A has C \ {j} promoted at g.
//
// The last block to finish then closes the stop: trace row, test count,
// the new cohort, CHECKFULLPASS (cohorts whose full pass is complete leave
// the window [head, tail)), |DASHED| and the loop test of Algorithm 2.
__global__ void __launch_bounds__(256) k_generate_finish(Lattice L, int slice_next) {
  pdl_wait();
  pdl_trigger();
  Ctrl *C = L.ctrl;
  // the loop state, read by one thread per CTA (every warp asking L2 for the
  // same line at once would serialise there); none of the fields the end of
  // the stop reads changes during this kernel except the candidate count,
  // which the last CTA's ticket returns
  __shared__ Ctrl s_c;
  if (threadIdx.x == 0) s_c = *C;
  __syncthreads();
  const uint32_t P = s_c.n_newbox, g = s_c.step, base = s_c.tail, l1 = L.l1;
  if (s_c.stall || s_c.done || s_c.error) return;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (slice_next)  // the columns of stop g+1 (count of stop g is complete)
    slice_block_warps(L, g + 1, tid >> 5, stride >> 5);
  if (L.vall && !L.events) {
    // bring the next stop's columns into L2 ahead of its count (one
    // 128-byte line per thread)
    const uint32_t *nv = vcols(L, g + 1);
    for (uint64_t i = tid * 32; i < L.vwords; i += stride * 32)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(nv + i));
  }
  const uint64_t total = (uint64_t)P * l1;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += stride) {
    gen_candidate(L, C, (uint32_t)(w / l1), (uint32_t)(w % l1), g, base);
  }
  // the event-driven loop's next cohort pass closes the stop (it reads the
  // final candidate count from the loop state)
  if (L.events) return;
  // the last CTA to finish closes the stop: its ticket (the high half of the
  // word whose low half every emitted candidate incremented, all of this
  // CTA's before the barrier) returns the stop's final candidate count
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long old = atomicAdd(&C->gen_ticket, 1ull << 32);
    if ((uint32_t)(old >> 32) == gridDim.x - 1) {
      const uint32_t n_gen = (uint32_t)old;
      // a slot past the capacity stalls the stop (ST_CAND, set by the CTA
      // that drew it); the host grows the store and re-runs generation
      if ((uint64_t)base + n_gen <= L.cap) {
        Ctrl c = s_c;
        c.gen_ticket = n_gen;
        finish_stop_with(L, C, c);
      }
    }
  }
}

cudaError_t launch_generate_finish(Lattice L, int grid, bool slice_next, cudaStream_t s) {
  return launch_k(k_generate_finish, grid, 256, 0, s, L, slice_next ? 1 : 0);
}

// --------------------------------------------------------------- output
// The boxes among records [0, tail), compacted in record order (so the
// first pass's pair records, which are in lexicographic rank order, come out
// in canonical order), in three launches: box counts per chunk of
// BOX_CHUNK records, an exclusive scan of those counts (one CTA), and a
// scatter of each chunk's box indices at its offset.
constexpr uint32_t BOX_CHUNK = 1024;
constexpr uint32_t BOX_THREADS = 256;

__global__ void __launch_bounds__(BOX_THREADS) k_box_count(Lattice L, uint32_t tail,
                                                           uint32_t *chunk_cnt) {
  const uint64_t c0 = (uint64_t)blockIdx.x * BOX_CHUNK;
  uint32_t n = 0;
  for (uint64_t c = c0 + threadIdx.x; c < c0 + BOX_CHUNK && c < tail; c += BOX_THREADS)
    n += L.cshape[c] == SH_BOX ? 1u : 0u;
  n = __reduce_add_sync(0xffffffffu, n);
  __shared__ uint32_t s_n[BOX_THREADS / 32];
  if ((threadIdx.x & 31) == 0) s_n[threadIdx.x >> 5] = n;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (uint32_t w = 0; w < BOX_THREADS / 32; ++w) t += s_n[w];
    chunk_cnt[blockIdx.x] = t;
  }
}

// In place: chunk_cnt[i] = boxes before chunk i; chunk_cnt[nchunks] = all.
__global__ void __launch_bounds__(1024) k_box_scan(uint32_t *chunk_cnt, uint32_t nchunks) {
  __shared__ uint32_t part[1024];
  const uint32_t per = (nchunks + 1023) / 1024;
  const uint32_t i0 = threadIdx.x * per;
  uint32_t sum = 0;
  for (uint32_t i = i0; i < i0 + per && i < nchunks; ++i) sum += chunk_cnt[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (uint32_t t = 0; t < 1024; ++t) { const uint32_t v = part[t]; part[t] = run; run += v; }
    chunk_cnt[nchunks] = run;
  }
  __syncthreads();
  uint32_t run = part[threadIdx.x];
  for (uint32_t i = i0; i < i0 + per && i < nchunks; ++i) {
    const uint32_t v = chunk_cnt[i];
    chunk_cnt[i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(BOX_THREADS) k_box_scatter(Lattice L, uint32_t tail,
                                                             const uint32_t *chunk_off,
                                                             uint32_t *out_idx) {
  __shared__ uint32_t s_w[BOX_THREADS / 32];
  __shared__ uint32_t s_base;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_base = chunk_off[blockIdx.x];
  const uint64_t c0 = (uint64_t)blockIdx.x * BOX_CHUNK;
  for (uint32_t r0 = 0; r0 < BOX_CHUNK; r0 += BOX_THREADS) {
    const uint64_t c = c0 + r0 + threadIdx.x;
    const bool box = c < tail && L.cshape[c] == SH_BOX;
    const uint32_t bal = __ballot_sync(0xffffffffu, box);
    __syncthreads();  // s_base and s_w of the previous round are settled
    if (lane == 0) s_w[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = s_base;
    for (uint32_t w = 0; w < warp; ++w) before += s_w[w];
    if (box) out_idx[before + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)c;
    __syncthreads();
    if (threadIdx.x == 0)
      for (uint32_t w = 0; w < BOX_THREADS / 32; ++w) s_base += s_w[w];
  }
}

cudaError_t launch_collect_boxes(Lattice L, uint32_t tail, uint32_t *chunk_cnt, uint32_t *out_idx,
                                 cudaStream_t s) {
  if (tail == 0) return cudaMemsetAsync(chunk_cnt, 0, 4, s);
  const uint32_t nchunks = (uint32_t)(((uint64_t)tail + BOX_CHUNK - 1) / BOX_CHUNK);
  k_box_count<<<nchunks, BOX_THREADS, 0, s>>>(L, tail, chunk_cnt);
  k_box_scan<<<1, 1024, 0, s>>>(chunk_cnt, nchunks);
  k_box_scatter<<<nchunks, BOX_THREADS, 0, s>>>(L, tail, chunk_cnt, out_idx);
  return cudaGetLastError();
}

uint32_t collect_chunks(uint32_t tail) {
  return (uint32_t)(((uint64_t)tail + BOX_CHUNK - 1) / BOX_CHUNK);
}

// Box q = record idx[q]: its size and support, and its items as original
// item ids (item_of[rank], ascending) in items[q][0 .. min(k, KRMAX)); with
// `masks` (itemsets longer than KRMAX exist) also its rank mask.
__global__ void k_gather_boxes(Lattice L, const uint32_t *idx, uint32_t cnt,
                               const uint32_t *item_of, uint32_t *out_k, uint32_t *out_supp,
                               uint32_t *items, uint64_t *masks) {
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = idx[q];
    const uint32_t k = L.ck[c];
    out_k[q] = k;
    out_supp[q] = L.csupp[c];
    const uint4 *rk4 = reinterpret_cast<const uint4 *>(L.cranks + (uint64_t)c * KRMAX);
    const uint4 ra = rk4[0], rb = rk4[1];
    const uint32_t rw[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
    const uint32_t kk = k < (uint32_t)KRMAX ? k : (uint32_t)KRMAX;
    for (uint32_t j = 0; j < kk; ++j)
      items[q * KRMAX + j] = item_of[(rw[j >> 1] >> (16 * (j & 1))) & 0xFFFFu];
    if (masks)
      for (uint32_t w = 0; w < L.wc; ++w) masks[q * L.wc + w] = L.cmask[(uint64_t)c * L.wc + w];
  }
}

cudaError_t launch_gather_boxes(Lattice L, const uint32_t *idx, uint32_t cnt,
                                const uint32_t *item_of, uint32_t *out_k, uint32_t *out_supp,
                                uint32_t *items, uint64_t *masks, cudaStream_t s) {
  if (cnt == 0) return cudaSuccess;
  const uint64_t want = ((uint64_t)cnt + 255) / 256;
  const int grid = (int)(want < 65535ull * 4 ? want : 65535ull * 4);
  k_gather_boxes<<<grid, 256, 0, s>>>(L, idx, cnt, item_of, out_k, out_supp, items, masks);
  return cudaGetLastError();
}

}  // namespace dic
