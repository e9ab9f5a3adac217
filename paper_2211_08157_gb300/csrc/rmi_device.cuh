// Device-side index lookups (hash table probe, learned-index evaluation and
// last-mile search), shared by the lookup kernels (index.cu, seed.cu) and the
// leaf-fitting kernels (rmi.cu). Both must route and predict
// with bit-identical FP32 arithmetic, so the operations are pinned with
// round-to-nearest intrinsics (no contraction freedom).
#pragma once
#include "common.cuh"

namespace god {

__device__ __forceinline__ float rmi_root_eval(const RmiRoot& R, uint64_t key) {
  const float x = __fmul_rn(__ull2float_rn(key - R.kmin), R.inv_span);
  float f = R.b2;
#pragma unroll
  for (int h = 0; h < kRootHidden; ++h) {
    const float a = fmaxf(__fmaf_rn(R.W1[h], x, R.b1[h]), 0.0f);
    f = __fmaf_rn(R.W2[h], a, f);
  }
  return f;
}

__device__ __forceinline__ uint32_t rmi_root_leaf(const RmiRoot& R, uint64_t key) {
  const float s = __fmul_rn(rmi_root_eval(R, key), (float)R.n_leaves);
  if (!(s > 0.0f)) return 0;
  if (s >= (float)R.n_leaves) return R.n_leaves - 1;
  return (uint32_t)floorf(s);
}

__device__ __forceinline__ int64_t rmi_leaf_pred(float slope, float icept, uint64_t base, uint64_t key) {
  const float d = __ll2float_rn((long long)(key - base));
  const float v = __fmaf_rn(slope, d, icept);
  if (!(v > -1.0e18f)) return INT64_MIN / 2;
  if (v > 1.0e18f) return INT64_MAX / 2;
  return (int64_t)floorf(v);
}

// Open-addressing probe: start | count << 32 of key, 0 when absent. Linear
// probing from the home slot key mod 2^lc; a slot holds the key's quotient
// key >> lc, its displacement d from the home slot and its rank in keys[]. The
// home slot is implied by the probe position, so (quotient, d) identifies the
// whole key and a match is exact.
__device__ __forceinline__ uint64_t ht_find(const DeviceIndex& di, uint64_t key) {
  const uint32_t lc = di.ht_lc, db = di.ht_db, rb = di.ht_rb;
  const uint64_t mask = (1ULL << lc) - 1, h = key & mask;
  const uint64_t q = key >> lc;
  const uint32_t qb = 64 - db - rb;            // quotient bits: keys below 2^(lc + qb) only
  if (lc + qb < 64 && (q >> qb) != 0) return 0;
  const uint64_t maxd = (1ULL << db) - 2;
  for (uint64_t d = 0; d <= maxd; ++d) {
    const uint64_t w = __ldg(di.ht + ((h + d) & mask));
    if (w == kEmptyKey) return 0;
    if ((w >> rb) == ((q << db) | d)) {
      const uint64_t r = w & ((1ULL << rb) - 1);
      const uint32_t s = __ldg(di.start + r), e = __ldg(di.start + r + 1);
      return (uint64_t)s | ((uint64_t)(e - s) << 32);
    }
  }
  return 0;
}

__device__ __forceinline__ uint64_t rmi_find(const DeviceIndex& di, const RmiRoot& R, uint64_t key) {
  if (key < R.kmin || key > R.kmax) return ht_find(di, key);
  const uint32_t leaf = rmi_root_leaf(R, key);
  const RmiLeaf L = di.leaves[leaf];
  const uint32_t eps = (uint32_t)(L.base_eps >> 56);
  if (eps > di.eps_max) return ht_find(di, key);
  const int64_t pred = rmi_leaf_pred(L.slope, L.icept, L.base_eps & ((1ULL << 56) - 1), key);
  int64_t lo = pred - (int64_t)eps, hi = pred + (int64_t)eps;
  if (lo < 0) lo = 0;
  if (hi > (int64_t)di.n_keys - 1) hi = (int64_t)di.n_keys - 1;
  while (lo <= hi) {  // last-mile binary search inside [pred - eps, pred + eps]
    const int64_t mid = (lo + hi) >> 1;
    const uint64_t km = __ldg(di.keys + mid);
    if (km == key) {
      const uint32_t s = __ldg(di.start + mid), e = __ldg(di.start + mid + 1);
      return (uint64_t)s | ((uint64_t)(e - s) << 32);
    }
    if (km < key) lo = mid + 1; else hi = mid - 1;
  }
  return 0;
}

}  // namespace god
