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

// Open-addressing probe: start | count << 32 of key, 0 when absent.
__device__ __forceinline__ uint64_t ht_find(const ulonglong2* __restrict__ ht, uint64_t mask, uint64_t key) {
  uint64_t slot = key & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const ulonglong2 e = __ldg(ht + slot);
    if (e.x == key) return e.y;
    if (e.x == kEmptyKey) return 0;
    slot = (slot + 1) & mask;
  }
  return 0;
}

__device__ __forceinline__ uint64_t rmi_find(const DeviceIndex& di, const RmiRoot& R, uint64_t key) {
  if (key < R.kmin || key > R.kmax) return ht_find(di.ht, di.ht_mask, key);
  const uint32_t leaf = rmi_root_leaf(R, key);
  const RmiLeaf L = di.leaves[leaf];
  const uint32_t eps = (uint32_t)(L.base_eps >> 56);
  if (eps > di.eps_max) return ht_find(di.ht, di.ht_mask, key);
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
