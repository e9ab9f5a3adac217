// Stable LSD radix sort of (u64 key, u64 value) pairs.
//
// Sec. 3.1 builds the seed index by appending (hash, location) pairs to an
// array and sorting it. Here that sort is a device-wide LSD radix sort. Each
// CTA of a fixed grid (a few per SM) owns one contiguous range of the input.
// A pass is three launches: every CTA counts the digits of its range, one CTA
// per digit turns that digit's counts into exclusive offsets over the ranges,
// and every CTA (adding the totals of the smaller digits) walks its range again in tiles of 2048 pairs, ranking each tile
// stably (warp ballots per digit bit give the lanes with an equal digit, then
// per-warp counters), staging it in shared memory in digit order and writing
// each digit run at its running offset. No CTA waits on another, so the time
// is one read for the counts plus one read and one write of the pairs. The
// input to the index sort is already in position order, so a stable sort by
// key alone yields (key, position).
#include <algorithm>

#include "common.cuh"

namespace god {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 8;                         // items per lane and tile
constexpr int kRsTile = kRsThreads * kRsRounds;      // 2048 items per tile
constexpr int kRsMaxBins = 256;
constexpr int kRsScanThreads = 1024;

__device__ __forceinline__ int range_of(uint64_t n, int G, int c, uint64_t* lo, uint64_t* hi) {
  const uint64_t tiles = (n + kRsTile - 1) / kRsTile;
  const uint64_t per = (tiles + G - 1) / G;              // tiles per range
  *lo = std::min<uint64_t>(n, (uint64_t)c * per * kRsTile);
  *hi = std::min<uint64_t>(n, (uint64_t)(c + 1) * per * kRsTile);
  return 0;
}

// cnt[d * G + c] = keys of range c with digit d.
__global__ void __launch_bounds__(kRsThreads) rs_count(const uint64_t* __restrict__ keys, uint64_t n, int shift,
                                                       int bits, uint32_t* __restrict__ cnt) {
  __shared__ uint32_t h[kRsWarps][kRsMaxBins];
  const int bins = 1 << bits;
  const int G = gridDim.x, c = blockIdx.x;
  const int wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * kRsMaxBins; i += kRsThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  uint64_t lo, hi;
  range_of(n, G, c, &lo, &hi);
  const uint64_t dmask = (uint64_t)bins - 1;
  for (uint64_t i = lo + threadIdx.x; i < hi; i += kRsThreads)
    atomicAdd(&h[wid][(int)((keys[i] >> shift) & dmask)], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < bins; d += kRsThreads) {
    uint32_t s = 0;
    for (int w = 0; w < kRsWarps; ++w) s += h[w][d];
    cnt[(uint64_t)d * G + c] = s;
  }
}

// Per digit (one CTA each): exclusive scan of the digit's counts over the
// ranges, in place, and the digit's total.
__global__ void __launch_bounds__(kRsScanThreads) rs_scan_rows(uint32_t* cnt, int G, uint32_t* tot) {
  __shared__ uint32_t warp_tot[kRsScanThreads / 32];
  __shared__ uint32_t carry;
  uint32_t* row = cnt + (uint64_t)blockIdx.x * G;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  for (int c0 = 0; c0 < G; c0 += kRsScanThreads) {
    const int c = c0 + threadIdx.x;
    const uint32_t v = c < G ? row[c] : 0;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      uint32_t t = warp_tot[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, t, d);
        if (lane >= d) t += y;
      }
      warp_tot[lane] = t;
    }
    __syncthreads();
    const uint32_t base = carry;
    if (c < G) row[c] = base + (wid ? warp_tot[wid - 1] : 0) + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry = base + warp_tot[kRsScanThreads / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

template <typename V>
__global__ void __launch_bounds__(kRsThreads, 4) rs_scatter(const uint64_t* __restrict__ keys_in,
                                                         const V* __restrict__ vals_in,
                                                         uint64_t* __restrict__ keys_out,
                                                         V* __restrict__ vals_out, uint64_t n, int shift,
                                                         int bits, const uint32_t* __restrict__ offs,
                                                         const uint32_t* __restrict__ tot) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(smem);          // kRsTile keys
  V* sv = reinterpret_cast<V*>(sk + kRsTile);                // kRsTile values
  uint32_t* whist = reinterpret_cast<uint32_t*>(sk + 2 * kRsTile);  // [warps][bins] (room for 8-byte values)
  uint32_t* dstart = whist + kRsWarps * kRsMaxBins;           // [bins] tile-local digit start
  uint32_t* run = dstart + kRsMaxBins;                        // [bins] running output offset
  __shared__ uint32_t warp_tot[kRsWarps];

  const int bins = 1 << bits;
  const uint32_t dmask = (uint32_t)bins - 1;
  const int G = gridDim.x, c = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  uint64_t lo, hi;
  range_of(n, G, c, &lo, &hi);
  {
    // digits below d over all ranges + digit d in the ranges before this one
    const int d = threadIdx.x;
    const uint32_t t = d < bins ? tot[d] : 0;
    uint32_t x = t;
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, s);
      if (lane >= s) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < wid; ++w) before += warp_tot[w];
    if (d < bins) run[d] = before + x - t + offs[(uint64_t)d * G + c];
    __syncthreads();
  }

  for (uint64_t tb = lo; tb < hi; tb += kRsTile) {
    for (int i = threadIdx.x; i < kRsWarps * kRsMaxBins; i += kRsThreads) whist[i] = 0;
    __syncthreads();
    const uint64_t warp_base = tb + (uint64_t)wid * (32 * kRsRounds);
    uint64_t k_reg[kRsRounds];
    uint32_t rank[kRsRounds];
    uint32_t* wh = whist + wid * kRsMaxBins;
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
      const uint64_t i = warp_base + (uint64_t)r * 32 + lane;
      const bool ok = i < hi;
      k_reg[r] = ok ? keys_in[i] : 0;
    }
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
      const uint64_t i = warp_base + (uint64_t)r * 32 + lane;
      const bool ok = i < hi;
      const uint32_t d = (uint32_t)(k_reg[r] >> shift) & dmask;
      // lanes holding the same digit: intersect the per-bit ballots
      unsigned peers = __ballot_sync(0xffffffffu, ok);
      for (int b = 0; b < bits; ++b) {
        const bool one = (d >> b) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, one);
        peers &= one ? bal : ~bal;
      }
      const uint32_t before = ok ? wh[d] : 0;
      __syncwarp();
      if (ok && (peers & lt_mask) == 0) wh[d] = before + __popc(peers);
      __syncwarp();
      rank[r] = before + __popc(peers & lt_mask);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, the tile's count, the tile-local start
    const int d = threadIdx.x;
    uint32_t cnt = 0;
    if (d < bins) {
      for (int w = 0; w < kRsWarps; ++w) {
        const uint32_t x = whist[w * kRsMaxBins + d];
        whist[w * kRsMaxBins + d] = cnt;
        cnt += x;
      }
    }
    {
      uint32_t x = cnt;
#pragma unroll
      for (int s = 1; s < 32; s <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, s);
        if (lane >= s) x += y;
      }
      if (lane == 31) warp_tot[wid] = x;
      __syncthreads();
      uint32_t before = 0;
      for (int w = 0; w < wid; ++w) before += warp_tot[w];
      if (d < bins) dstart[d] = before + x - cnt;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
      const uint64_t i = warp_base + (uint64_t)r * 32 + lane;
      if (i < hi) {
        const uint32_t dg = (uint32_t)(k_reg[r] >> shift) & dmask;
        const uint32_t q = dstart[dg] + whist[wid * kRsMaxBins + dg] + rank[r];
        sk[q] = k_reg[r];
        sv[q] = vals_in[i];
      }
    }
    __syncthreads();
    const uint32_t valid = (uint32_t)std::min<uint64_t>(kRsTile, hi - tb);
    for (uint32_t q = threadIdx.x; q < valid; q += kRsThreads) {
      const uint64_t key = sk[q];
      const uint32_t dg = (uint32_t)(key >> shift) & dmask;
      const uint64_t dst = (uint64_t)run[dg] + (q - dstart[dg]);
      keys_out[dst] = key;
      vals_out[dst] = sv[q];
    }
    __syncthreads();
    if (d < bins) run[d] += cnt;
  }
}

size_t scatter_smem() {
  return (size_t)kRsTile * 16 + (size_t)kRsWarps * kRsMaxBins * 4 + 2 * kRsMaxBins * 4;
}

template <typename V>
int radix_sort_impl(uint64_t* keys, V* vals, uint64_t n, int key_bits, cudaStream_t st) {
  if (n <= 1 || key_bits <= 0) return GOD_OK;
  if (n >= (1ULL << 32)) {
    set_error("radix sort: at most 2^32 - 1 pairs");
    return GOD_EINVAL;
  }
  int passes = (key_bits + 7) / 8;
  if (passes & 1) ++passes;  // even pass count: the result lands back in the caller's buffers
  const int bits = (key_bits + passes - 1) / passes;
  const int bins = 1 << bits;
  const size_t smem = scatter_smem();
  GOD_CK(cudaFuncSetAttribute(rs_scatter<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GOD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rs_scatter<V>, kRsThreads, smem));
  const uint64_t tiles = (n + kRsTile - 1) / kRsTile;
  const int G = (int)std::max<uint64_t>(1, std::min<uint64_t>(tiles, (uint64_t)num_sms() * std::max(per_sm, 1)));
  const uint64_t m = (uint64_t)bins * G;
  DBuf<uint64_t> k2;
  DBuf<V> v2;
  DBuf<uint32_t> cnt, tot;
  GOD_TRY(k2.alloc(n, st));
  GOD_TRY(v2.alloc(n, st));
  GOD_TRY(cnt.alloc(m, st));
  GOD_TRY(tot.alloc(bins, st));
  uint64_t *ki = keys, *ko = k2.p;
  V *vi = vals, *vo = v2.p;
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = ps * bits;
    GOD_LAUNCH(rs_count, (unsigned)G, kRsThreads, 0, st, ki, n, shift, bits, cnt.p);
    GOD_LAUNCH(rs_scan_rows, (unsigned)bins, kRsScanThreads, 0, st, cnt.p, G, tot.p);
    GOD_LAUNCH(rs_scatter<V>, (unsigned)G, kRsThreads, smem, st, ki, vi, ko, vo, n, shift, bits, cnt.p, tot.p);
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  // passes is even: ki == keys
  return GOD_OK;
}

}  // namespace

int radix_sort_pairs(uint64_t* keys, uint64_t* vals, uint64_t n, int key_bits, cudaStream_t st) {
  return radix_sort_impl(keys, vals, n, key_bits, st);
}
int radix_sort_pairs32(uint64_t* keys, uint32_t* vals, uint64_t n, int key_bits, cudaStream_t st) {
  return radix_sort_impl(keys, vals, n, key_bits, st);
}

}  // namespace god
