// Bucket sort of the index's (key, value) pairs: one pass by the key's top b
// bits, then one shared-memory sort per bucket.
//
// The index keys are hash values, uniform over [0, 2^key_bits), and every
// value (pos << 1 | z) is distinct. So the pairs sorted by (key, value) are
// the pairs sorted by the 64-bit composite (key's low key_bits - b bits) <<
// vbits | value inside each bucket of the key's top b bits, and the order in
// which pairs reach a bucket does not matter: the scatter takes its slots
// with atomics (no stable ranking), and each bucket is then sorted on chip.
// With b chosen for about 2048 pairs per bucket, the pairs cross DRAM twice
// (bucket scatter, bucket sort) instead of once per 7-bit digit (six times
// for 42-bit keys). Buckets past 8192 pairs (repeated keys) are sorted in
// 8192-pair chunks merged by merge-path passes in a global buffer.
// Same result as a stable sort by key of pairs in value order (the input).
#include <algorithm>

#include "common.cuh"

namespace god {
namespace {

constexpr int kBkThreads = 512;
constexpr uint32_t kBkCap = 8192;          // pairs sorted in shared memory at once
constexpr uint64_t kBkTarget = 2048;       // mean pairs per bucket

__global__ void bk_count(const uint64_t* __restrict__ keys, uint64_t n, int shift, uint32_t* __restrict__ cnt) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + (keys[i] >> shift), 1u);
}

template <typename V>
__global__ void bk_scatter(const uint64_t* __restrict__ keys, const V* __restrict__ vals, uint64_t n, int shift,
                           int vbits, unsigned long long* __restrict__ cursor, uint64_t* __restrict__ comp) {
  const uint64_t lowmask = (1ull << shift) - 1;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
    const unsigned long long at = atomicAdd(cursor + (k >> shift), 1ull);
    if (at < n) comp[at] = ((k & lowmask) << vbits) | (uint64_t)vals[i];
  }
}

__device__ void bitonic_smem64(uint64_t* s, uint32_t n_pad) {
  for (uint32_t kk = 2; kk <= n_pad; kk <<= 1) {
    for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint64_t x = s[i], y = s[ixj];
          if ((x > y) == ((i & kk) == 0)) {
            s[i] = y;
            s[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Loads comp[lo, lo + m) (m <= kBkCap) into s and sorts it.
__device__ void load_sort(const uint64_t* comp, uint64_t lo, uint32_t m, uint64_t* s) {
  uint32_t n_pad = 1;
  while (n_pad < m) n_pad <<= 1;
  for (uint32_t q = threadIdx.x; q < n_pad; q += blockDim.x) s[q] = q < m ? comp[lo + q] : ~0ull;
  __syncthreads();
  bitonic_smem64(s, n_pad);
}

__device__ void merge_path64(const uint64_t* x, uint64_t nx, const uint64_t* y, uint64_t ny, uint64_t* o) {
  constexpr int IPT = 8;
  const uint64_t total = nx + ny;
  for (uint64_t d0 = (uint64_t)threadIdx.x * IPT; d0 < total; d0 += (uint64_t)blockDim.x * IPT) {
    uint64_t lo = d0 > ny ? d0 - ny : 0, hi = d0 < nx ? d0 : nx;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (x[mid] < y[d0 - 1 - mid]) lo = mid + 1;
      else hi = mid;
    }
    uint64_t i = lo, j = d0 - lo;
    for (int t = 0; t < IPT && d0 + t < total; ++t) {
      if (j >= ny || (i < nx && x[i] < y[j])) o[d0 + t] = x[i++];
      else o[d0 + t] = y[j++];
    }
  }
}

// A CTA per bucket (grid-stride): sort the bucket's composites and write the
// pairs back in order. comp2 is scratch of the same size as comp.
template <typename V>
__global__ void __launch_bounds__(kBkThreads) bk_sort(uint64_t* comp, uint64_t* comp2,
                                                      const unsigned long long* __restrict__ start, uint64_t n_buckets,
                                                      uint64_t n, int shift, int vbits, uint64_t* __restrict__ keys,
                                                      V* __restrict__ vals) {
  extern __shared__ __align__(16) uint64_t s[];
  const uint64_t vmask = vbits >= 64 ? ~0ull : ((1ull << vbits) - 1);
  for (uint64_t bkt = blockIdx.x; bkt < n_buckets; bkt += gridDim.x) {
    const uint64_t lo = start[bkt], hi = start[bkt + 1];
    if (hi <= lo || hi > n) continue;   // (only after a scan that gave up; reported by bk_starts)
    const uint64_t m = hi - lo;
    const uint64_t* res;
    if (m <= kBkCap) {
      load_sort(comp, lo, (uint32_t)m, s);
      res = s;
    } else {
      // sorted runs of kBkCap, then merge passes (ping-pong in comp / comp2)
      for (uint64_t c0 = 0; c0 < m; c0 += kBkCap) {
        const uint32_t cm = (uint32_t)std::min<uint64_t>(kBkCap, m - c0);
        load_sort(comp, lo + c0, cm, s);
        for (uint32_t q = threadIdx.x; q < cm; q += blockDim.x) comp2[lo + c0 + q] = s[q];
        __syncthreads();
      }
      uint64_t* x = comp2 + lo;
      uint64_t* y = comp + lo;
      for (uint64_t run = kBkCap; run < m; run <<= 1) {
        for (uint64_t j = 0; j < m; j += 2 * run) {
          const uint64_t na = std::min<uint64_t>(run, m - j);
          const uint64_t nb = j + run < m ? std::min<uint64_t>(run, m - j - run) : 0;
          merge_path64(x + j, na, x + j + na, nb, y + j);
        }
        __syncthreads();
        uint64_t* t = x;
        x = y;
        y = t;
      }
      res = x;
    }
    for (uint64_t q = threadIdx.x; q < m; q += blockDim.x) {
      const uint64_t c = res[q];
      keys[lo + q] = (bkt << shift) | (c >> vbits);
      vals[lo + q] = (V)(c & vmask);
    }
    __syncthreads();
  }
}

// Bucket starts and scatter cursors from the scanned counts; err = 1 when the
// scan's total is not n (a look-back wait gave up).
__global__ void bk_starts(uint64_t nb, uint64_t n, const uint64_t* __restrict__ off,
                          unsigned long long* __restrict__ start, unsigned long long* __restrict__ cursor, int* err) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= nb; i += (uint64_t)gridDim.x * blockDim.x) {
    start[i] = off[i];
    if (i < nb) cursor[i] = off[i];
    if (i == nb && off[i] != n) atomicExch(err, 1);
  }
}

inline unsigned grid_for(uint64_t n, int per, unsigned cap_mult) {
  uint64_t b = (n + per - 1) / per;
  b = std::max<uint64_t>(b, 1);
  return (unsigned)std::min<uint64_t>(b, (uint64_t)num_sms() * cap_mult);
}

template <typename V>
int bucket_sort_impl(uint64_t* keys, V* vals, uint64_t n, int key_bits, int vbits, int* d_err, cudaStream_t st,
                     bool* done) {
  *done = false;
  if (n < 4 * kBkTarget) return GOD_OK;
  int b = 1;
  while (b < 24 && (n >> b) > kBkTarget) ++b;
  b = std::min(b, key_bits);
  const int shift = key_bits - b;
  if (vbits >= 64 || shift + vbits > 64) return GOD_OK;   // the composite does not fit: sorted by digits instead
  const uint64_t nb = 1ull << b;
  DBuf<uint32_t> cnt;
  DBuf<uint64_t> off, comp, comp2;
  DBuf<unsigned long long> start, cursor;
  GOD_TRY(cnt.alloc(nb, st));
  GOD_TRY(off.alloc(nb + 1, st));
  GOD_TRY(start.alloc(nb + 1, st));
  GOD_TRY(cursor.alloc(nb, st));
  GOD_TRY(comp.alloc(n, st));
  GOD_TRY(comp2.alloc(n, st));
  GOD_CK(cudaMemsetAsync(cnt.p, 0, nb * 4, st));
  GOD_LAUNCH(bk_count, grid_for(n, 256, 16), 256, 0, st, keys, n, shift, cnt.p);
  GOD_TRY(exclusive_scan_u32(cnt.p, off.p, nb, st));
  GOD_LAUNCH(bk_starts, grid_for(nb + 1, 256, 16), 256, 0, st, nb, n, off.p, start.p, cursor.p, d_err);
  GOD_LAUNCH(bk_scatter<V>, grid_for(n, 256, 16), 256, 0, st, keys, vals, n, shift, vbits, cursor.p, comp.p);
  const size_t smem = kBkCap * sizeof(uint64_t);
  GOD_CK(cudaFuncSetAttribute(bk_sort<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)std::min<uint64_t>(nb, (uint64_t)num_sms() * 3);
  GOD_LAUNCH(bk_sort<V>, grid, kBkThreads, smem, st, comp.p, comp2.p, start.p, nb, n, shift, vbits, keys, vals);
  *done = true;
  return GOD_OK;
}

}  // namespace

int bucket_sort_pairs(uint64_t* keys, uint64_t* vals, uint64_t n, int key_bits, int vbits, int* d_err,
                      cudaStream_t st, bool* done) {
  return bucket_sort_impl(keys, vals, n, key_bits, vbits, d_err, st, done);
}
int bucket_sort_pairs32(uint64_t* keys, uint32_t* vals, uint64_t n, int key_bits, int vbits, int* d_err,
                        cudaStream_t st, bool* done) {
  return bucket_sort_impl(keys, vals, n, key_bits, vbits, d_err, st, done);
}

}  // namespace god
