// Association rules from the frequent itemsets: the second subtask of
// Section 1 (the paper leaves its definition to its reference [1]; the
// textbook one is used). For every frequent Z with |Z| >= 2 and every
// non-empty proper subset X of Z, X -> Z \ X holds when its confidence
// supp(Z) / supp(X) is at least num / den, compared exactly in integers as
// supp(Z) * den >= num * supp(X). Every subset of a frequent itemset is
// frequent, so supp(X) is looked up among the itemsets themselves.
//
//   k_rules_insert  open-addressing table over the itemsets' masks
//   k_rules_eval    one thread per (Z, split code): bit b of the code picks
//                   the b-th item of Z (ascending) for X; X's hash and key
//                   are derived word by word from Z and the code without
//                   materialising X; rules are appended with an atomic
//                   cursor (the host sorts them canonically)
#include <cstdint>
#include <cuda_runtime.h>

#include "dic_internal.cuh"
#include "lattice_device.cuh"

namespace dic {

struct RuleSet {
  const uint64_t *masks;        // [count][W] itemsets (item p = bit p%64 of word p/64)
  const uint32_t *k;            // [count] sizes
  const uint32_t *supp;         // [count] supports
  const uint64_t *work_prefix;  // [count + 1] exclusive prefix of 2^k - 2 (k >= 2, else 0)
  uint32_t *hslot;              // [hcap] itemset index + 1, 0 = empty
  uint64_t count;
  uint32_t W;
  uint32_t hcap;                // power of two >= 2 * count
};

// Word i of X = the items of Z's word i whose order among Z's items (bits
// before word i: `before`) is selected by `code`.
__device__ __forceinline__ uint64_t split_word(uint64_t zw, uint32_t before, uint32_t code) {
  uint64_t x = 0;
  uint32_t t = before;
  for (uint64_t y = zw; y; y &= y - 1, ++t)
    if ((code >> t) & 1u) x |= y & (~y + 1);  // lowest set bit of y
  return x;
}

__global__ void k_rules_insert(RuleSet R, uint32_t *err) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < R.count;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t slot = hslot_of(mask_hash_sum(R.masks + i * R.W, R.W), R.hcap);
    bool placed = false;
    for (uint32_t probe = 0; probe < R.hcap && !placed; ++probe) {
      placed = atomicCAS(&R.hslot[slot], 0u, (uint32_t)i + 1) == 0u;
      slot = (slot + 1) & (R.hcap - 1);
    }
    if (!placed) atomicOr(err, 2u);  // table full: a sizing error
  }
}

__global__ void k_rules_eval(RuleSet R, uint32_t num, uint32_t den, uint64_t total,
                             unsigned long long *cursor, uint32_t *out_z, uint32_t *out_code,
                             uint32_t *out_sx, uint32_t *err) {
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total;
       w += (uint64_t)gridDim.x * blockDim.x) {
    // the itemset Z whose range of split codes holds w
    uint64_t lo = 0, hi = R.count;  // work_prefix[lo] <= w < work_prefix[hi]
    while (hi - lo > 1) {
      const uint64_t mid = (lo + hi) / 2;
      if (R.work_prefix[mid] <= w) lo = mid; else hi = mid;
    }
    const uint64_t zi = lo;
    const uint32_t code = (uint32_t)(w - R.work_prefix[zi]) + 1u;  // 1 .. 2^k - 2
    const uint64_t *Z = R.masks + zi * R.W;
    // hash of X, from Z and the code
    uint64_t sum = 0;
    uint32_t before = 0;
    for (uint32_t i = 0; i < R.W; ++i) {
      sum += hterm(split_word(Z[i], before, code), i);
      before += __popcll(Z[i]);
    }
    uint32_t slot = hslot_of(sum, R.hcap), found = 0;
    for (uint32_t probe = 0; probe < R.hcap; ++probe) {
      const uint32_t v = R.hslot[slot];
      if (v == 0) break;
      const uint64_t *key = R.masks + (uint64_t)(v - 1) * R.W;
      bool eq = true;
      before = 0;
      for (uint32_t i = 0; i < R.W && eq; ++i) {
        eq = key[i] == split_word(Z[i], before, code);
        before += __popcll(Z[i]);
      }
      if (eq) { found = v; break; }
      slot = (slot + 1) & (R.hcap - 1);
    }
    if (!found) {  // a subset of a frequent itemset is missing from the input
      atomicOr(err, 1u);
      continue;
    }
    const uint64_t sz = R.supp[zi], sx = R.supp[found - 1];
    if (sz * den >= (uint64_t)num * sx) {
      const unsigned long long pos = atomicAdd(cursor, 1ull);
      if (pos < total) {  // (cannot fail: one slot per split)
        out_z[pos] = (uint32_t)zi;
        out_code[pos] = code;
        out_sx[pos] = (uint32_t)sx;
      }
    }
  }
}

static int grid_for(uint64_t items) {
  const uint64_t want = (items + 255) / 256;
  return (int)(want < 1 ? 1 : (want > 65535ull * 8 ? 65535ull * 8 : want));
}

cudaError_t launch_rules(const uint64_t *masks, const uint32_t *k, const uint32_t *supp,
                         const uint64_t *work_prefix, uint32_t *hslot, uint64_t count,
                         uint32_t W, uint32_t hcap, uint32_t num, uint32_t den, uint64_t total,
                         unsigned long long *cursor, uint32_t *out_z, uint32_t *out_code,
                         uint32_t *out_sx, uint32_t *err, cudaStream_t s) {
  RuleSet R{masks, k, supp, work_prefix, hslot, count, W, hcap};
  k_rules_insert<<<grid_for(count), 256, 0, s>>>(R, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || total == 0) return e;
  k_rules_eval<<<grid_for(total), 256, 0, s>>>(R, num, den, total, cursor, out_z, out_code,
                                               out_sx, err);
  return cudaGetLastError();
}

}  // namespace dic
