// Device-wide exclusive prefix sums in one pass (decoupled look-back).
//
// Tiles of 4096 values take numbers from a ticket in the order they start,
// sum their values, publish the tile sum, and warp 0 adds the sums of the
// tiles before it (reading back until a tile that has published its
// inclusive prefix), so every tile waits only on tiles already running. Each
// wait is bounded; a wait that gives up poisons the total (out[n] = ~0),
// which every caller reads back to size its next buffers, so the failure
// surfaces as an impossible size rather than a silent wrong offset.
#include "common.cuh"

namespace god {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr uint64_t kFlagAgg = 1ULL << 62;
constexpr uint64_t kFlagIncl = 2ULL << 62;
constexpr uint64_t kValMask = (1ULL << 62) - 1;
constexpr uint32_t kScanSpinLimit = 1u << 22;

__device__ __forceinline__ uint64_t ld_acquire_u64(const unsigned long long* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* excl) {
  __shared__ uint64_t warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint64_t t = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, t, d);
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

__device__ __forceinline__ uint64_t warp_sum(uint64_t v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// Warp-wide inclusive scan.
__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t x, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  return x;
}

// Each warp takes 512 consecutive values of the tile as 16 rows of 32 (every
// load and store coalesced), scanning row by row.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) scan_onepass(const T* __restrict__ in, uint64_t n,
                                                             uint64_t* __restrict__ out,
                                                             unsigned long long* status, unsigned int* ticket) {
  __shared__ uint32_t s_tile;
  __shared__ uint64_t s_prefix;
  __shared__ bool s_bad;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  const int lane0 = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t base = (uint64_t)tile * kScanTile + (uint64_t)wid * (32 * kScanItems) + lane0;
  uint64_t v[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint64_t j = base + 32 * i;
    v[i] = j < n ? (uint64_t)in[j] : 0;
  }
  uint64_t s = 0;                                  // this warp's running total over rows
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint64_t x = warp_incl_scan(v[i], lane0);
    v[i] = s + x - v[i];                           // exclusive within the warp's 512 values
    s += __shfl_sync(0xffffffffu, x, 31);
  }
  uint64_t excl;                                   // warps before this one (lane values equal)
  const uint64_t total = block_exclusive_scan(lane0 == 0 ? s : 0, &excl);
  excl = __shfl_sync(0xffffffffu, excl, 0);
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    uint64_t prefix = 0;
    bool bad = false;
    if (tile == 0) {
      if (lane == 0) st_release_u64(status, kFlagIncl | total);
    } else {
      if (lane == 0) st_release_u64(status + tile, kFlagAgg | total);
      int64_t pbase = (int64_t)tile - 1;
      uint32_t spins = 0;
      while (true) {
        const int64_t idx = pbase - lane;
        uint64_t st = idx >= 0 ? ld_acquire_u64(status + idx) : kFlagIncl;
        while (!__all_sync(0xffffffffu, (st & (kFlagAgg | kFlagIncl)) != 0)) {
          if (++spins > kScanSpinLimit) {
            bad = true;
            if (!(st & (kFlagAgg | kFlagIncl))) st = kFlagIncl;
            break;
          }
          __nanosleep(32);
          if (!(st & (kFlagAgg | kFlagIncl))) st = ld_acquire_u64(status + idx);
        }
        const unsigned im = __ballot_sync(0xffffffffu, (st & kFlagIncl) != 0);
        if (im) {
          const int first = __ffs(im) - 1;          // nearest earlier tile with its inclusive prefix
          prefix += warp_sum(lane <= first ? (st & kValMask) : 0);
          break;
        }
        prefix += warp_sum(st & kValMask);
        pbase -= 32;
      }
      bad = __any_sync(0xffffffffu, bad);
      if (lane == 0) st_release_u64(status + tile, kFlagIncl | (prefix + total));
    }
    if (lane == 0) {
      s_prefix = prefix;
      s_bad = bad;
    }
  }
  __syncthreads();
  const uint64_t add = s_prefix + excl;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint64_t j = base + 32 * i;
    if (j < n) out[j] = add + v[i];
  }
  if ((uint64_t)(tile + 1) * kScanTile >= n && threadIdx.x == 0) out[n] = s_bad ? ~0ULL : s_prefix + total;
}

template <typename T>
int scan_launch(const T* in, uint64_t* out, uint64_t n, uint64_t* ws, cudaStream_t st) {
  if (n == 0) {
    GOD_CK(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
    return GOD_OK;
  }
  const uint64_t nt = (n + kScanTile - 1) / kScanTile;
  GOD_CK(cudaMemsetAsync(ws, 0, (size_t)(nt + 1) * sizeof(uint64_t), st));
  GOD_LAUNCH(scan_onepass<T>, (unsigned)nt, kScanThreads, 0, st, in, n, out,
             reinterpret_cast<unsigned long long*>(ws), reinterpret_cast<unsigned int*>(ws + nt));
  return GOD_OK;
}

template <typename T>
int scan_impl(const T* in, uint64_t* out, uint64_t n, cudaStream_t st) {
  DBuf<uint64_t> ws;
  GOD_TRY(ws.alloc(scan_ws_words(n), st));
  return scan_launch(in, out, n, ws.p, st);
}

}  // namespace

// tile status words + the tile ticket
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
