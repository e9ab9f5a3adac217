// Device-wide exclusive prefix sums (reduce-then-scan, deterministic).
#include "common.cuh"

namespace god {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ uint64_t load_as_u64(const T* in, uint64_t i, uint64_t n) {
  return i < n ? (uint64_t)in[i] : 0ULL;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* excl) {
  __shared__ uint64_t warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint64_t y = __shfl_up_sync(0xffffffffu, t, d);
      if (lane >= d) t += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  const uint64_t before = wid ? warp_tot[wid - 1] : 0;
  *excl = before + x - v;
  const uint64_t total = warp_tot[kScanThreads / 32 - 1];
  __syncthreads();
  return total;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) tile_sums_kernel(const T* in, uint64_t n, uint64_t* sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) s += load_as_u64(in, base + (uint64_t)i * kScanThreads + threadIdx.x, n);
  uint64_t excl;
  const uint64_t tot = block_exclusive_scan(s, &excl);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single CTA: exclusive scan of the tile sums, in place; sums[nt] = total.
__global__ void __launch_bounds__(kScanThreads) scan_sums_kernel(uint64_t* sums, uint64_t nt) {
  uint64_t carry = 0;
  for (uint64_t base = 0; base < nt; base += kScanThreads) {
    const uint64_t i = base + threadIdx.x;
    const uint64_t v = i < nt ? sums[i] : 0;
    uint64_t excl;
    const uint64_t tot = block_exclusive_scan(v, &excl);
    if (i < nt) sums[i] = carry + excl;
    carry += tot;
  }
  if (threadIdx.x == 0) sums[nt] = carry;
}

template <typename T>
__global__ void __launch_bounds__(kScanThreads) tile_scan_kernel(const T* in, uint64_t n, const uint64_t* sums,
                                                                  uint64_t* out, uint64_t nt) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint64_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = load_as_u64(in, base + i, n);
    s += v[i];
  }
  uint64_t excl;
  block_exclusive_scan(s, &excl);
  uint64_t run = sums[blockIdx.x] + excl;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (blockIdx.x == nt - 1 && threadIdx.x == 0) out[n] = sums[nt];
}

template <typename T>
int scan_launch(const T* in, uint64_t* out, uint64_t n, uint64_t* sums, cudaStream_t st) {
  if (n == 0) {
    GOD_CK(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
    return GOD_OK;
  }
  const uint64_t nt = (n + kScanTile - 1) / kScanTile;
  GOD_LAUNCH(tile_sums_kernel<T>, (unsigned)nt, kScanThreads, 0, st, in, n, sums);
  GOD_LAUNCH(scan_sums_kernel, 1, kScanThreads, 0, st, sums, nt);
  GOD_LAUNCH(tile_scan_kernel<T>, (unsigned)nt, kScanThreads, 0, st, in, n, sums, out, nt);
  return GOD_OK;
}

template <typename T>
int scan_impl(const T* in, uint64_t* out, uint64_t n, cudaStream_t st) {
  DBuf<uint64_t> sums;
  GOD_TRY(sums.alloc(scan_ws_words(n), st));
  return scan_launch(in, out, n, sums.p, st);
}

}  // namespace

uint64_t scan_ws_words(uint64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

int exclusive_scan_u32(const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st) {
  return scan_impl(in, out, n, st);
}
int exclusive_scan_u32_ws(const uint32_t* in, uint64_t* out, uint64_t n, uint64_t* ws, cudaStream_t st) {
  return scan_launch(in, out, n, ws, st);
}
int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t st) {
  return scan_impl(in, out, n, st);
}

}  // namespace god
