// Device-side index lookups (hash table probe, learned-index evaluation and
// last-mile search), shared by the lookup kernels (index.cu, seed.cu) and the
// leaf-fitting kernels (rmi.cu). Both must route and predict
// with bit-identical FP32 arithmetic, so the operations are pinned with
// round-to-nearest intrinsics (no contraction freedom).
#pragma once
#include "common.cuh"

namespace god {

// Root model at the key: the piece holding x (bisection over the hinge
// points) and one multiply-add.
__device__ __forceinline__ float rmi_root_eval(const RmiRoot& R, uint64_t key) {
  const float x = __fmul_rn(__ull2float_rn(key - R.kmin), R.inv_span);
  int i = 0;
#pragma unroll
  for (int step = kRootHidden / 2; step > 0; step >>= 1)
    if (R.hx[i + step - 1] <= x) i += step;
  if (R.hx[i] <= x) ++i;   // i = hinges <= x (0..32)
  return __fmaf_rn(R.A[i], x, R.C[i]);
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

// Open-addressing probe. Linear probing from the home slot key mod 2^lc; a
// slot holds the key's quotient key >> lc, its displacement d from the home
// slot and a field: the key's (start, count) in the entry array when those
// fit (payload slots, one memory access per lookup), else its rank in keys[]
// (the offsets then come from start[rank], start[rank + 1]). The home slot is
// implied by the probe position, so (quotient, d) identifies the whole key
// and a match is exact.
constexpr uint64_t kNoRank = ~0ULL;

__device__ __forceinline__ uint64_t ht_home_word(const DeviceIndex& di, uint64_t key) {
  return __ldg(di.ht + (key & ((1ULL << di.ht_lc) - 1)));
}

// Slot field of key (kNoRank when absent), given the word at its home slot
// (loaded by the caller, so that several probes can be in flight).
__device__ __forceinline__ uint64_t ht_field(const DeviceIndex& di, uint64_t key, uint64_t w0) {
  const uint32_t lc = di.ht_lc, db = di.ht_db, rb = di.ht_rb;
  const uint64_t mask = (1ULL << lc) - 1, h = key & mask;
  const uint64_t q = key >> lc;
  const uint32_t qb = 64 - db - rb;            // quotient bits: keys below 2^(lc + qb) only
  if (lc + qb < 64 && (q >> qb) != 0) return kNoRank;
  const uint64_t maxd = (1ULL << db) - 2;
  uint64_t w = w0;
  for (uint64_t d = 0; d <= maxd; ++d) {
    if (d) w = __ldg(di.ht + ((h + d) & mask));
    if (w == kEmptyKey) return kNoRank;
    if ((w >> rb) == ((q << db) | d)) return w & ((1ULL << rb) - 1);
  }
  return kNoRank;
}

// start | count << 32 of a key rank (0 for kNoRank).
__device__ __forceinline__ uint64_t rank_payload(const DeviceIndex& di, uint64_t r) {
  if (r == kNoRank) return 0;
  const uint32_t s = __ldg(di.start + r), e = __ldg(di.start + r + 1);
  return (uint64_t)s | ((uint64_t)(e - s) << 32);
}

// start | count << 32 of a slot field (0 for kNoRank).
__device__ __forceinline__ uint64_t field_payload(const DeviceIndex& di, uint64_t f) {
  if (di.ht_cb == 0 || f == kNoRank) return rank_payload(di, f);
  return (f >> di.ht_cb) | ((f & ((1ULL << di.ht_cb) - 1)) << 32);
}

// start | count << 32 of key, 0 when absent.
__device__ __forceinline__ uint64_t ht_find(const DeviceIndex& di, uint64_t key) {
  return field_payload(di, ht_field(di, key, ht_home_word(di, key)));
}

// Learned-index lookup in steps, so that a caller can keep several keys in
// flight: rmi_leaf_of (root model, no memory access), then the leaf load, then
// rmi_rank_in_leaf (last-mile search in [pred - eps, pred + eps]). Keys outside
// the modelled range or in a leaf whose bound exceeds eps_max go to the hash
// table.
__device__ __forceinline__ bool rmi_in_range(const RmiRoot& R, uint64_t key) {
  return key >= R.kmin && key <= R.kmax;
}

// Rank of key in keys[] inside the leaf's window [pred - eps, pred + eps],
// kNoRank when absent. A window of at most 8 keys is read at once
// (independent loads) and scanned; wider ones are bisected.
template <int N>
__device__ __forceinline__ uint64_t key_scan(const DeviceIndex& di, int64_t lo, int64_t hi, uint64_t key) {
  uint64_t km[N];
#pragma unroll
  for (int t = 0; t < N; ++t) km[t] = lo + t <= hi ? __ldg(di.keys + lo + t) : ~0ULL;
  uint64_t r = kNoRank;
#pragma unroll
  for (int t = 0; t < N; ++t)
    if (lo + t <= hi && km[t] == key) r = (uint64_t)(lo + t);
  return r;
}

__device__ __forceinline__ uint64_t rmi_rank_in_leaf(const DeviceIndex& di, const RmiLeaf& L, uint64_t key) {
  const uint32_t eps = (uint32_t)(L.base_eps >> 56);
  const int64_t pred = rmi_leaf_pred(L.slope, L.icept, L.base_eps & ((1ULL << 56) - 1), key);
  int64_t lo = pred - (int64_t)eps, hi = pred + (int64_t)eps;
  if (lo < 0) lo = 0;
  if (hi > (int64_t)di.n_keys - 1) hi = (int64_t)di.n_keys - 1;
  if (hi - lo < 8) return key_scan<8>(di, lo, hi, key);   // one width: lanes of a warp stay together
  while (lo <= hi) {
    const int64_t mid = (lo + hi) >> 1;
    const uint64_t km = __ldg(di.keys + mid);
    if (km == key) return (uint64_t)mid;
    if (km < key) lo = mid + 1; else hi = mid - 1;
  }
  return kNoRank;
}

__device__ __forceinline__ uint64_t rmi_find(const DeviceIndex& di, const RmiRoot& R, uint64_t key) {
  if (!rmi_in_range(R, key)) return ht_find(di, key);
  const RmiLeaf L = di.leaves[rmi_root_leaf(R, key)];
  if ((uint32_t)(L.base_eps >> 56) > di.eps_max) return ht_find(di, key);
  return rank_payload(di, rmi_rank_in_leaf(di, L, key));
}

}  // namespace god
