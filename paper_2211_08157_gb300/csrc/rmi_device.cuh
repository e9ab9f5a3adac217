// Device-side evaluation of the learned index, shared by the lookup kernels
// (index.cu) and the leaf-fitting kernels (rmi.cu). Both must route and predict
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

}  // namespace god
