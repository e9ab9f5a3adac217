// Stable LSD radix sort of (u64 key, u64 value) pairs.
//
// Sec. 3.1 builds the seed index by appending (hash, location) pairs to an
// array and sorting it. Here that sort is a device-wide LSD radix sort; each
// pass is an upsweep (per-tile digit histograms), a digit-major exclusive scan,
// and a downsweep that ranks keys stably inside the tile (warp match_any +
// per-warp counters), stages the tile in shared memory in digit order and then
// writes each digit run contiguously. The input to the index sort is already
// in position order, so a stable sort by key alone yields (key, position).
#include <algorithm>

#include "common.cuh"

namespace god {
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;                        // items per lane
constexpr int kRsTile = kRsThreads * kRsRounds;      // 4096 items per CTA
constexpr int kRsMaxBins = 256;

__global__ void __launch_bounds__(kRsThreads) rs_upsweep(const uint64_t* keys, uint64_t n, int shift, int bits,
                                                         uint32_t* hist, uint32_t n_tiles) {
  __shared__ uint32_t h[kRsMaxBins];
  const int bins = 1 << bits;
  for (int i = threadIdx.x; i < bins; i += kRsThreads) h[i] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kRsTile;
  const uint64_t dmask = (uint64_t)bins - 1;
#pragma unroll 4
  for (int r = 0; r < kRsRounds; ++r) {
    const uint64_t i = base + (uint64_t)r * kRsThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & dmask], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < bins; d += kRsThreads) hist[(uint64_t)d * n_tiles + blockIdx.x] = h[d];
}

__global__ void __launch_bounds__(kRsThreads) rs_downsweep(const uint64_t* keys_in, const uint64_t* vals_in,
                                                           uint64_t* keys_out, uint64_t* vals_out, uint64_t n,
                                                           int shift, int bits, const uint64_t* offsets,
                                                           uint32_t n_tiles) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(smem);          // kRsTile keys
  uint64_t* sv = sk + kRsTile;                               // kRsTile values
  uint32_t* whist = reinterpret_cast<uint32_t*>(sv + kRsTile);  // [warps][bins]
  uint32_t* dstart = whist + kRsWarps * kRsMaxBins;           // [bins] tile-local digit start
  uint64_t* gbase = reinterpret_cast<uint64_t*>(dstart + kRsMaxBins);  // [bins] global start

  const int bins = 1 << bits;
  const uint32_t dmask = (uint32_t)bins - 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRsWarps * kRsMaxBins; i += kRsThreads) whist[i] = 0;
  __syncthreads();

  const uint64_t tile_base = (uint64_t)blockIdx.x * kRsTile;
  const uint64_t warp_base = tile_base + (uint64_t)wid * (32 * kRsRounds);
  uint64_t k_reg[kRsRounds];
  uint32_t rank[kRsRounds];
  uint32_t* wh = whist + wid * kRsMaxBins;
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const uint64_t i = warp_base + (uint64_t)r * 32 + lane;
    const bool ok = i < n;
    k_reg[r] = ok ? keys_in[i] : 0;
    const uint32_t d = ok ? (uint32_t)(k_reg[r] >> shift) & dmask : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = ok ? wh[d] : 0;
    __syncwarp();
    if (ok && (peers & lt_mask) == 0) wh[d] = before + __popc(peers);
    __syncwarp();
    rank[r] = before + __popc(peers & lt_mask);
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, tile total
  for (int d = threadIdx.x; d < bins; d += kRsThreads) {
    uint32_t run = 0;
    for (int w = 0; w < kRsWarps; ++w) {
      const uint32_t c = whist[w * kRsMaxBins + d];
      whist[w * kRsMaxBins + d] = run;
      run += c;
    }
    dstart[d] = run;  // tile total for now
    gbase[d] = offsets[(uint64_t)d * n_tiles + blockIdx.x];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int d = 0; d < bins; ++d) { const uint32_t c = dstart[d]; dstart[d] = run; run += c; }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRsRounds; ++r) {
    const uint64_t i = warp_base + (uint64_t)r * 32 + lane;
    if (i < n) {
      const uint32_t d = (uint32_t)(k_reg[r] >> shift) & dmask;
      const uint32_t q = dstart[d] + whist[wid * kRsMaxBins + d] + rank[r];
      sk[q] = k_reg[r];
      sv[q] = vals_in[i];
    }
  }
  __syncthreads();
  const uint64_t valid = n > tile_base ? std::min<uint64_t>(kRsTile, n - tile_base) : 0;
  for (uint32_t q = threadIdx.x; q < valid; q += kRsThreads) {
    const uint64_t key = sk[q];
    const uint32_t d = (uint32_t)(key >> shift) & dmask;
    const uint64_t dst = gbase[d] + (q - dstart[d]);
    keys_out[dst] = key;
    vals_out[dst] = sv[q];
  }
}

size_t downsweep_smem() {
  return (size_t)kRsTile * 16 + (size_t)kRsWarps * kRsMaxBins * 4 + kRsMaxBins * 4 + kRsMaxBins * 8;
}

}  // namespace

int radix_sort_pairs(uint64_t* keys, uint64_t* vals, uint64_t n, int key_bits, cudaStream_t st) {
  if (n <= 1 || key_bits <= 0) return GOD_OK;
  int passes = (key_bits + 7) / 8;
  if (passes & 1) ++passes;  // even pass count: the result lands back in the caller's buffers
  const int bits = (key_bits + passes - 1) / passes;
  const uint64_t n_tiles64 = (n + kRsTile - 1) / kRsTile;
  if (n_tiles64 > 0xFFFFFFFFull) return GOD_EINVAL;
  const uint32_t n_tiles = (uint32_t)n_tiles64;
  DBuf<uint64_t> k2, v2, offs;
  DBuf<uint32_t> hist;
  GOD_TRY(k2.alloc(n, st));
  GOD_TRY(v2.alloc(n, st));
  const uint64_t nh = (uint64_t)(1 << bits) * n_tiles;
  GOD_TRY(hist.alloc(nh, st));
  GOD_TRY(offs.alloc(nh + 1, st));
  const size_t smem = downsweep_smem();
  GOD_CK(cudaFuncSetAttribute(rs_downsweep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  uint64_t *ki = keys, *vi = vals, *ko = k2.p, *vo = v2.p;
  for (int ps = 0; ps < passes; ++ps) {
    const int shift = ps * bits;
    GOD_LAUNCH(rs_upsweep, n_tiles, kRsThreads, 0, st, ki, n, shift, bits, hist.p, n_tiles);
    GOD_TRY(exclusive_scan_u32(hist.p, offs.p, nh, st));
    GOD_LAUNCH(rs_downsweep, n_tiles, kRsThreads, smem, st, ki, vi, ko, vo, n, shift, bits, offs.p, n_tiles);
    std::swap(ki, ko);
    std::swap(vi, vo);
  }
  // passes is even: ki == keys
  return GOD_OK;
}

}  // namespace god
