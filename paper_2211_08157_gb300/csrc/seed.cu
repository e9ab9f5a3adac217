// Batched pattern alignment (Sec. 3.2) and compressed seeding (Sec. 3.3).
//
// All reads of a batch go through one pass of the sketch kernel as segments
// (read, shift) of its virtual stream:
//  * PA pass: every read at every shift s < p. With a limit t on the
//    minimizers used per shift and odd k, only a prefix of t*w + w + k - 2
//    patterned bases is sketched: windows starting before t*w are complete,
//    disjoint windows [0, w), [w, 2w), ... each hold a minimizer, so an N-free
//    prefix already contains the first t minimizers of the whole read. A read
//    whose prefix holds an N is re-run at full length (fallback pass).
//  * The read's alignment index a = the shift whose first t minimizers have the
//    largest summed index count (smallest shift on ties, 0 when all are 0).
//  * Seeding pass: the minimizers of the read at shift a. When the PA pass saw
//    the whole read at shift a they are reused; otherwise the read is sketched
//    again at shift a, full length.
//  * Every seeding minimizer whose key is kept in the index yields one anchor
//    per index entry; anchors are counted per read, offsets scanned, and each
//    read's anchors are produced and sorted in on-chip memory in one step
//    (a thread per read for lists of at most 16, a warp per read for short
//    lists, a CTA per read with a shared-memory radix sort for long ones; lists
//    past 4096 anchors are sorted in chunks merged by merge-path passes).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "rmi_device.cuh"

namespace god {
namespace {

constexpr int kT = 256;
constexpr uint32_t kSrcPA = 0, kSrcFB = 1, kSrcP2 = 2;
constexpr int kSmallCap = 128;          // anchors per read for the warp path
constexpr int kMedThreads = 128;
constexpr int kWarpCap = 512;           // anchors per read for the warp bitonic path
constexpr int kMedCap = 1024;           // anchors per read for the medium CTA path
constexpr int kLargeThreads = 256;
constexpr int kLargeCap = 4096;         // anchors sorted in shared memory at once
constexpr int kLargeRounds = kLargeCap / kLargeThreads;

inline unsigned grid_for(uint64_t n, int per = kT, unsigned cap_mult = 32) {
  uint64_t b = (n + per - 1) / per;
  b = std::max<uint64_t>(b, 1);
  return (unsigned)std::min<uint64_t>(b, (uint64_t)num_sms() * cap_mult);
}

struct RecSet {
  const uint32_t* pz;       // (read position << 1) | z of each record
  const uint64_t* sc;       // lookup result: start | count << 32
  const uint64_t* seg_off;  // first record of each segment
  const uint32_t* seg_cnt;  // records of each segment
};
struct RecSets {
  RecSet s[3];
};
// Constant indices only: a runtime index into a parameter array would copy it
// to local memory.
__device__ __forceinline__ RecSet pick_set(const RecSets& S, uint32_t k) {
  return k == 0 ? S.s[0] : (k == 1 ? S.s[1] : S.s[2]);
}

constexpr int kTinyCap = 16;            // anchors per read for the thread path

// Appends i to list (unordered) with one atomic per warp.
__device__ __forceinline__ void warp_append(bool f, uint32_t i, uint32_t* list, unsigned long long* counter) {
  const unsigned am = __activemask();
  const unsigned bal = __ballot_sync(am, f);
  if (!bal) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(am) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(bal));
  base = __shfl_sync(am, base, leader);
  if (f) list[base + __popc(bal & ((1u << lane) - 1u))] = i;
}

__global__ void make_pa_segments(const uint64_t* __restrict__ offs, uint32_t n, PatternInfo P, uint32_t cap,
                                 SegDesc* __restrict__ segs, uint32_t* __restrict__ vlen, int* err,
                                 uint32_t* max_m) {
  uint32_t mlen = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = offs[i];
    uint64_t e = offs[i + 1];
    if (e < b || e - b >= (1ull << 31)) {
      atomicExch(err, 1);
      e = b;
    }
    const uint64_t len = e - b;
    for (int s = 0; s < P.p; ++s) {
      const uint64_t g = i * P.p + s;
      const uint64_t m = patterned_len(P, len, s);
      const uint32_t mm = (uint32_t)std::min<uint64_t>(m, cap);
      segs[g] = SegDesc{b, mm, (uint32_t)i, (uint32_t)s, m > cap ? kSegCapped : 0u};
      vlen[g] = mm + 1;
      mlen = mm > mlen ? mm : mlen;
    }
  }
  const unsigned am = __activemask();
  mlen = __reduce_max_sync(am, mlen);
  if ((int)(threadIdx.x & 31) == __ffs(am) - 1) atomicMax(max_m, mlen);
}

// Segments at full length for listed reads: all shifts (fallback PA) or the
// chosen shift only (seeding pass).
__global__ void make_list_segments(const uint64_t* __restrict__ offs, const uint32_t* __restrict__ list, uint32_t nl,
                                   PatternInfo P, int all_shifts, const uint32_t* __restrict__ shift,
                                   SegDesc* __restrict__ segs, uint32_t* __restrict__ vlen, uint32_t* max_m) {
  uint32_t mlen = 0;
  for (uint64_t li = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; li < nl; li += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = list[li];
    const uint64_t b = offs[i], len = offs[i + 1] - b;
    if (all_shifts) {
      for (int s = 0; s < P.p; ++s) {
        const uint64_t m = patterned_len(P, len, s);
        segs[li * P.p + s] = SegDesc{b, (uint32_t)m, i, (uint32_t)s, 0u};
        vlen[li * P.p + s] = (uint32_t)m + 1;
        mlen = (uint32_t)m > mlen ? (uint32_t)m : mlen;
      }
    } else {
      const uint32_t s = shift[i];
      const uint64_t m = patterned_len(P, len, s);
      segs[li] = SegDesc{b, (uint32_t)m, i, s, 0u};
      vlen[li] = (uint32_t)m + 1;
      mlen = (uint32_t)m > mlen ? (uint32_t)m : mlen;
    }
  }
  const unsigned am = __activemask();
  mlen = __reduce_max_sync(am, mlen);
  if ((int)(threadIdx.x & 31) == __ffs(am) - 1) atomicMax(max_m, mlen);
}

// Sum of index counts over a segment's first t records (t = 0: all) and over
// all of its records.
__device__ __forceinline__ void shift_sums(const RecSet& S, uint64_t g, uint32_t t, uint64_t* sum_t, uint64_t* sum_all) {
  const uint64_t beg = S.seg_off[g];
  const uint32_t c = S.seg_cnt[g];
  uint64_t a = 0, b = 0;
  for (uint32_t j = 0; j < c; ++j) {
    const uint64_t v = S.sc[beg + j] >> 32;
    b += v;
    if (!t || j < t) a += v;
  }
  *sum_t = a;
  *sum_all = b;
}

// Pattern alignment over the PA pass: one thread per read. The chosen shift's
// whole-segment count is the read's anchor count when that segment was not a
// prefix; otherwise the read joins the seeding-pass list (or the fallback list
// when its prefix held an N).
__global__ void pa_select(uint32_t n, int p, uint32_t t, const SegDesc* __restrict__ segs, RecSet S,
                          const uint32_t* __restrict__ need_full, uint32_t* __restrict__ shift,
                          uint32_t* __restrict__ src, uint32_t* __restrict__ seed_seg, uint64_t* __restrict__ read_cnt,
                          uint32_t* __restrict__ fb_list, uint32_t* __restrict__ p2_list,
                          unsigned long long* __restrict__ counts) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    bool fb = false, p2 = false;
    if (need_full[i]) {
      fb = true;
      src[i] = kSrcFB;
    } else {
      uint64_t best = 0, all_a = 0;
      uint32_t a = 0;
      for (int s = 0; s < p; ++s) {
        uint64_t st, sa;
        shift_sums(S, i * p + s, t, &st, &sa);
        if (s == 0 || st > best) { best = st; a = (uint32_t)s; all_a = sa; }
      }
      shift[i] = a;
      seed_seg[i] = (uint32_t)(i * p + a);
      p2 = segs[i * p + a].flags & kSegCapped;
      src[i] = p2 ? kSrcP2 : kSrcPA;
      if (!p2) read_cnt[i] = all_a;
    }
    warp_append(fb, (uint32_t)i, fb_list, counts + 0);
    warp_append(p2, (uint32_t)i, p2_list, counts + 1);
  }
}

// Pattern alignment of fallback reads over their full-length segments.
__global__ void pa_select_list(const uint32_t* __restrict__ list, uint32_t nl, int p, uint32_t t, RecSet S,
                               uint32_t* __restrict__ shift, uint32_t* __restrict__ seed_seg,
                               uint64_t* __restrict__ read_cnt) {
  for (uint64_t li = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; li < nl; li += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t best = 0, all_a = 0;
    uint32_t a = 0;
    for (int s = 0; s < p; ++s) {
      uint64_t st, sa;
      shift_sums(S, li * p + s, t, &st, &sa);
      if (s == 0 || st > best) { best = st; a = (uint32_t)s; all_a = sa; }
    }
    const uint32_t i = list[li];
    shift[i] = a;
    seed_seg[i] = (uint32_t)(li * p + a);
    read_cnt[i] = all_a;
  }
}

__global__ void set_seed_seg_list(const uint32_t* __restrict__ list, uint32_t nl, uint32_t* __restrict__ seed_seg) {
  for (uint64_t li = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; li < nl; li += (uint64_t)gridDim.x * blockDim.x)
    seed_seg[list[li]] = (uint32_t)li;
}

// Anchors of the listed reads = sum of index counts of their seeding-pass
// minimizers (segment li of the set belongs to list[li]; warp per read).
__global__ void count_anchors_list(const uint32_t* __restrict__ list, uint32_t nl, RecSet S,
                                   uint64_t* __restrict__ read_cnt) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t li = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; li < nl; li += warps) {
    const uint64_t beg = S.seg_off[li];
    const uint32_t c = S.seg_cnt[li];
    uint64_t sum = 0;
    for (uint32_t j = lane; j < c; j += 32) sum += S.sc[beg + j] >> 32;
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (lane == 0) read_cnt[list[li]] = sum;
  }
}

// Reads by anchor-list length: tiny (thread path), small (warp path), large
// (CTA path). Lists are unordered; every read writes its own output range.
// counts: [tiny, small, warp, medium, large, huge reads, chunks of the huge
// reads (kLargeCap anchors each), most chunks of one read].
__global__ void classify_reads(uint32_t n, const uint64_t* __restrict__ read_off, uint32_t* __restrict__ tiny,
                               uint32_t* __restrict__ small, uint32_t* __restrict__ warpl,
                               uint32_t* __restrict__ medium, uint32_t* __restrict__ large,
                               uint32_t* __restrict__ huge, unsigned long long* __restrict__ counts) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t c = read_off[i + 1] - read_off[i];
    warp_append(c > 0 && c <= kTinyCap, (uint32_t)i, tiny, counts + 0);
    warp_append(c > kTinyCap && c <= kSmallCap, (uint32_t)i, small, counts + 1);
    warp_append(c > kSmallCap && c <= kWarpCap, (uint32_t)i, warpl, counts + 2);
    warp_append(c > kWarpCap && c <= kMedCap, (uint32_t)i, medium, counts + 3);
    warp_append(c > kMedCap && c <= kLargeCap, (uint32_t)i, large, counts + 4);
    warp_append(c > kLargeCap, (uint32_t)i, huge, counts + 5);
    if (c > kLargeCap) {
      const unsigned long long ch = (c + kLargeCap - 1) / kLargeCap;
      atomicAdd(counts + 6, ch);
      atomicMax(counts + 7, ch);
    }
  }
}

// One task per kLargeCap-anchor tile of every huge read: (huge-list index <<
// 32) | tile. The chunk sorts and every merge level take the same tiles.
__global__ void huge_tasks(const uint32_t* __restrict__ huge, uint32_t n_huge, const uint64_t* __restrict__ read_off,
                           uint64_t* __restrict__ tasks, unsigned long long* __restrict__ ctr) {
  for (uint32_t li = blockIdx.x * blockDim.x + threadIdx.x; li < n_huge; li += gridDim.x * blockDim.x) {
    const uint32_t i = huge[li];
    const uint64_t ch = (read_off[i + 1] - read_off[i] + kLargeCap - 1) / kLargeCap;
    const unsigned long long b = atomicAdd(ctr, ch);
    for (uint64_t c = 0; c < ch; ++c) tasks[b + c] = ((uint64_t)li << 32) | c;
  }
}

__device__ __forceinline__ uint64_t anchor_key(uint64_t entry, uint32_t read_pos, uint32_t z) {
  return ((entry >> 1) << 32) | ((uint64_t)read_pos << 1) | ((entry & 1u) ^ z);
}

__device__ __forceinline__ void store_anchor(god_anchor* out, uint32_t read, uint64_t key) {
  uint4 v;
  v.x = read;
  v.y = (uint32_t)(key >> 1) & 0x7FFFFFFFu;
  v.z = (uint32_t)(key >> 32);
  v.w = (uint32_t)(key & 1u);
  __stcs(reinterpret_cast<uint4*>(out), v);   // streamed: keep the index entries in L2
}

// Tiny anchor lists (<= 16): one thread per read gathers them into registers
// (compile-time slots) and sorts them with a 16-wide bitonic network.
__device__ __forceinline__ void cswap(uint64_t& a, uint64_t& b, bool up) {
  const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
  a = up ? lo : hi;
  b = up ? hi : lo;
}

// Records whose loads a tiny-list thread keeps in flight (2,000,000 x 150 bp
// reads: 1, 2, 4, 8 records took 0.38, 0.32, 0.29, 0.33 ms per batch).
constexpr int kFillBatch = 4;

__global__ void __launch_bounds__(kT) fill_sort_tiny(RecSets sets, const uint32_t* __restrict__ src,
                                                     const uint32_t* __restrict__ seed_seg,
                                                     const uint64_t* __restrict__ read_off,
                                                     const uint32_t* __restrict__ list, uint32_t nl,
                                                     const uint64_t* __restrict__ ent, god_anchor* __restrict__ out) {
  for (uint64_t li = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; li < nl; li += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = list[li];
    const uint64_t off = read_off[i];
    const uint32_t n = (uint32_t)(read_off[i + 1] - off);
    const RecSet S = pick_set(sets, src[i]);
    const uint32_t g = seed_seg[i];
    const uint64_t beg = S.seg_off[g];
    const uint32_t cnt = S.seg_cnt[g];
    uint64_t v[kTinyCap];
#pragma unroll
    for (int q = 0; q < kTinyCap; ++q) v[q] = ~0ULL;
    uint32_t fill = 0;
    // kFillBatch records at a time: their lookups, then their positions and
    // first entries (most keys occur once), so the dependent loads overlap
    for (uint32_t r0 = 0; r0 < cnt; r0 += kFillBatch) {
      uint64_t sc[kFillBatch], e0[kFillBatch];
      uint32_t pzv[kFillBatch];
#pragma unroll
      for (int u = 0; u < kFillBatch; ++u) sc[u] = r0 + u < cnt ? S.sc[beg + r0 + u] : 0;
#pragma unroll
      for (int u = 0; u < kFillBatch; ++u) {
        const bool hit = (sc[u] >> 32) != 0;
        pzv[u] = hit ? S.pz[beg + r0 + u] : 0u;
        e0[u] = hit ? __ldg(ent + (uint32_t)sc[u]) : 0;
      }
#pragma unroll
      for (int u = 0; u < kFillBatch; ++u) {
        const uint32_t c = (uint32_t)(sc[u] >> 32);
        for (uint32_t e = 0; e < c; ++e, ++fill) {
          const uint64_t en = e ? __ldg(ent + (uint32_t)sc[u] + e) : e0[u];
          const uint64_t key = anchor_key(en, pzv[u] >> 1, pzv[u] & 1u);
#pragma unroll
          for (int q = 0; q < kTinyCap; ++q) v[q] = (q == (int)fill) ? key : v[q];
        }
      }
    }
#pragma unroll
    for (int kk = 2; kk <= kTinyCap; kk <<= 1) {
#pragma unroll
      for (int j = kk >> 1; j > 0; j >>= 1) {
#pragma unroll
        for (int q = 0; q < kTinyCap; ++q) {
          const int r2 = q ^ j;
          if (r2 > q) cswap(v[q], v[r2], (q & kk) == 0);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kTinyCap; ++q)
      if (q < (int)n) store_anchor(out + off + q, i, v[q]);
  }
}

// Short anchor lists: one warp per read builds the list in shared memory and
// places every anchor at its rank (keys are distinct within a read).
__global__ void __launch_bounds__(kT) fill_sort_small(RecSets sets, const uint32_t* __restrict__ src,
                                                      const uint32_t* __restrict__ seed_seg,
                                                      const uint64_t* __restrict__ read_off,
                                                      const uint32_t* __restrict__ list, uint32_t nl,
                                                      const uint64_t* __restrict__ ent, god_anchor* __restrict__ out) {
  __shared__ uint64_t buf[kT / 32][kSmallCap];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t* B = buf[wid];
  const uint64_t warps = (uint64_t)gridDim.x * (kT / 32);
  for (uint64_t li = (blockIdx.x * (uint64_t)kT + threadIdx.x) / 32; li < nl; li += warps) {
    const uint32_t i = list[li];
    const uint64_t off = read_off[i];
    const uint32_t n = (uint32_t)(read_off[i + 1] - off);
    const RecSet S = pick_set(sets, src[i]);
    const uint32_t g = seed_seg[i];
    const uint64_t beg = S.seg_off[g];
    const uint32_t cnt = S.seg_cnt[g];
    uint32_t base = 0;
    for (uint32_t r0 = 0; r0 < cnt; r0 += 32) {
      const uint32_t r = r0 + lane;
      uint32_t c = 0, start = 0, pos = 0, z = 0;
      if (r < cnt) {
        const uint64_t sc = S.sc[beg + r];
        c = (uint32_t)(sc >> 32);
        start = (uint32_t)sc;
        if (c) {
          const uint32_t pzv = S.pz[beg + r];
          pos = pzv >> 1;
          z = pzv & 1u;
        }
      }
      uint32_t incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
      }
      // the 32 records' entries expanded by the whole warp (a lane finds the
      // record of entry q by a binary search over the lanes' exclusive counts)
      const uint32_t ex = incl - c;
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      for (uint32_t q0 = 0; q0 < tot; q0 += 32) {
        const uint32_t q = q0 + lane;
        int L = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t e = __shfl_sync(0xffffffffu, ex, L + step);
          if (e <= q) L += step;
        }
        const uint32_t eL = __shfl_sync(0xffffffffu, ex, L);
        const uint32_t sL = __shfl_sync(0xffffffffu, start, L);
        const uint32_t pL = __shfl_sync(0xffffffffu, pos, L);
        const uint32_t zL = __shfl_sync(0xffffffffu, z, L);
        if (q < tot) B[base + q] = anchor_key(__ldg(ent + sL + (q - eL)), pL, zL);
      }
      base += tot;
    }
    __syncwarp();
    for (uint32_t e = lane; e < n; e += 32) {
      const uint64_t key = B[e];
      uint32_t rank = 0;
      for (uint32_t f = 0; f < n; ++f) rank += B[f] < key;
      store_anchor(out + off + rank, i, key);
    }
    __syncwarp();
  }
}

// ---- CTA helpers for long lists
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* total, uint32_t* warp_buf) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x / 32;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) warp_buf[wid] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int w = 0; w < nw; ++w) { const uint32_t c = warp_buf[w]; warp_buf[w] = run; run += c; }
    warp_buf[nw] = run;
  }
  __syncthreads();
  const uint32_t r = warp_buf[wid] + x - v;
  *total = warp_buf[nw];
  __syncthreads();
  return r;
}

// Writes anchor keys with list index in [lo, hi) to dst[idx - lo].
__device__ void fill_range(const RecSet& S, uint64_t beg, uint32_t cnt, const uint64_t* __restrict__ ent, uint64_t lo,
                           uint64_t hi, uint64_t* dst, uint32_t* warp_buf) {
  uint64_t base = 0;
  for (uint32_t r0 = 0; r0 < cnt; r0 += blockDim.x) {
    const uint32_t r = r0 + threadIdx.x;
    uint32_t c = 0, start = 0, pos = 0, z = 0;
    if (r < cnt) {
      const uint64_t sc = S.sc[beg + r];
      c = (uint32_t)(sc >> 32);
      start = (uint32_t)sc;
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan_u32(c, &tot, warp_buf);
    if (base + tot > lo && base < hi && c) {
      const uint64_t a0 = base + ex;
      const uint64_t e_lo = a0 < lo ? lo - a0 : 0;
      const uint64_t e_hi = a0 + c > hi ? (hi > a0 ? hi - a0 : 0) : c;
      if (e_lo < e_hi) {
        const uint32_t pzv = S.pz[beg + r];
        pos = pzv >> 1;
        z = pzv & 1u;
        for (uint64_t e = e_lo; e < e_hi; ++e) dst[a0 + e - lo] = anchor_key(__ldg(ent + start + e), pos, z);
      }
    }
    base += tot;
    if (base >= hi) break;
  }
}

__device__ void key_field_bits(const uint64_t* s, uint32_t n, int* lo_bits, int* hi_bits, uint32_t* warp_buf);
__device__ uint64_t* cta_radix_sort(uint64_t* a, uint64_t* b, uint32_t n, int lo_bits, int hi_bits,
                                    uint32_t* whist, uint32_t* dstart, uint32_t* warp_buf);

__device__ void bitonic_sort_smem(uint64_t* s, uint32_t n_pad) {
  for (uint32_t k = 2; k <= n_pad; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint64_t a = s[i], b = s[ixj];
          const bool up = (i & k) == 0;
          if ((a > b) == up) { s[i] = b; s[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

// Anchor lists of kSmallCap < n <= kWarpCap (short reads on repeat-rich
// references): one warp per read, 4 KB of keys in shared memory, the
// records' entries expanded by the whole warp (a lane finds the record of
// entry q by a binary search over the lanes' exclusive counts), and a
// bitonic network over the padded list with warp barriers only (no CTA-wide
// barrier per stage, so the warps of an SM interleave freely).
__global__ void __launch_bounds__(kT) fill_sort_warp(RecSets sets, const uint32_t* __restrict__ src,
                                                     const uint32_t* __restrict__ seed_seg,
                                                     const uint64_t* __restrict__ read_off,
                                                     const uint32_t* __restrict__ list, uint32_t nl,
                                                     const uint64_t* __restrict__ ent, god_anchor* __restrict__ out) {
  __shared__ uint64_t buf[kT / 32][kWarpCap];
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t* B = buf[wid];
  const uint64_t warps = (uint64_t)gridDim.x * (kT / 32);
  for (uint64_t li = (blockIdx.x * (uint64_t)kT + threadIdx.x) / 32; li < nl; li += warps) {
    const uint32_t i = list[li];
    const uint64_t off = read_off[i];
    const uint32_t n = (uint32_t)(read_off[i + 1] - off);
    const RecSet S = pick_set(sets, src[i]);
    const uint32_t g = seed_seg[i];
    const uint64_t beg = S.seg_off[g];
    const uint32_t cnt = S.seg_cnt[g];
    uint32_t base = 0;
    for (uint32_t r0 = 0; r0 < cnt; r0 += 32) {
      const uint32_t r = r0 + lane;
      uint32_t c = 0, start = 0, pzv = 0;
      if (r < cnt) {
        const uint64_t sc = S.sc[beg + r];
        c = (uint32_t)(sc >> 32);
        start = (uint32_t)sc;
        if (c) pzv = S.pz[beg + r];
      }
      uint32_t incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += y;
      }
      const uint32_t ex = incl - c;
      const uint32_t tot = __shfl_sync(FULL, incl, 31);
      for (uint32_t q0 = 0; q0 < tot; q0 += 32) {   // warp-uniform trip count
        const uint32_t q = q0 + lane;
        int L = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t e = __shfl_sync(FULL, ex, L + step);
          if (e <= q) L += step;
        }
        const uint32_t eL = __shfl_sync(FULL, ex, L);
        const uint32_t sL = __shfl_sync(FULL, start, L);
        const uint32_t pL = __shfl_sync(FULL, pzv, L);
        if (q < tot) B[base + q] = anchor_key(__ldg(ent + sL + (q - eL)), pL >> 1, pL & 1u);
      }
      base += tot;
    }
    uint32_t n_pad = 32;
    while (n_pad < n) n_pad <<= 1;
    for (uint32_t q = n + lane; q < n_pad; q += 32) B[q] = ~0ULL;
    __syncwarp();
    for (uint32_t kk = 2; kk <= n_pad; kk <<= 1) {
      for (uint32_t jj = kk >> 1; jj > 0; jj >>= 1) {
        for (uint32_t t = lane; t < n_pad / 2; t += 32) {
          const uint32_t lo = ((t & ~(jj - 1)) << 1) | (t & (jj - 1)), hi = lo + jj;
          const uint64_t a = B[lo], b = B[hi];
          if ((a > b) == ((lo & kk) == 0)) {
            B[lo] = b;
            B[hi] = a;
          }
        }
        __syncwarp();
      }
    }
    for (uint32_t q = lane; q < n; q += 32) store_anchor(out + off + q, i, B[q]);
    __syncwarp();
  }
}

// Medium anchor lists (kWarpCap < n <= kMedCap; short reads on repeat-rich
// references): a 128-thread CTA per read, the keys in 8 KB of shared memory
// (16 CTAs fit an SM, where the 256-thread large path with its 74 KB fit 3 and
// spent its time waiting at barriers), entries expanded by all threads (a
// thread finds the record of entry q by a binary search over the records'
// exclusive counts, so one repeat key with many entries does not leave one
// thread loading them all), a bitonic network over the padded list.
__global__ void __launch_bounds__(kMedThreads) fill_sort_medium(RecSets sets, const uint32_t* __restrict__ src,
                                                                const uint32_t* __restrict__ seed_seg,
                                                                const uint64_t* __restrict__ read_off,
                                                                const uint32_t* __restrict__ list, uint32_t nl,
                                                                const uint64_t* __restrict__ ent,
                                                                god_anchor* __restrict__ out) {
  __shared__ uint64_t s[kMedCap];
  __shared__ uint32_t s_ex[kMedThreads], s_start[kMedThreads], s_pz[kMedThreads];
  __shared__ uint32_t warp_buf[kMedThreads / 32 + 1];
  for (uint32_t li = blockIdx.x; li < nl; li += gridDim.x) {
    const uint32_t i = list[li];
    const uint64_t off = read_off[i];
    const uint32_t n = (uint32_t)(read_off[i + 1] - off);
    const RecSet S = pick_set(sets, src[i]);
    const uint32_t g = seed_seg[i];
    const uint64_t beg = S.seg_off[g];
    const uint32_t cnt = S.seg_cnt[g];
    uint32_t base = 0;
    for (uint32_t r0 = 0; r0 < cnt; r0 += kMedThreads) {
      const uint32_t r = r0 + threadIdx.x;
      uint32_t c = 0, start = 0, pzv = 0;
      if (r < cnt) {
        const uint64_t sc = S.sc[beg + r];
        c = (uint32_t)(sc >> 32);
        start = (uint32_t)sc;
        if (c) pzv = S.pz[beg + r];
      }
      uint32_t tot;
      const uint32_t ex = block_excl_scan_u32(c, &tot, warp_buf);
      s_ex[threadIdx.x] = ex;
      s_start[threadIdx.x] = start;
      s_pz[threadIdx.x] = pzv;
      __syncthreads();
      for (uint32_t q = threadIdx.x; q < tot; q += kMedThreads) {
        uint32_t j = 0;   // last record with s_ex[j] <= q
#pragma unroll
        for (uint32_t step = kMedThreads / 2; step > 0; step >>= 1)
          if (s_ex[j + step] <= q) j += step;
        const uint32_t pj = s_pz[j];
        s[base + q] = anchor_key(__ldg(ent + s_start[j] + (q - s_ex[j])), pj >> 1, pj & 1u);
      }
      __syncthreads();
      base += tot;
    }
    uint32_t n_pad = 1;
    while (n_pad < n) n_pad <<= 1;
    for (uint32_t q = n + threadIdx.x; q < n_pad; q += kMedThreads) s[q] = ~0ULL;
    __syncthreads();
    bitonic_sort_smem(s, n_pad);
    for (uint32_t q = threadIdx.x; q < n; q += kMedThreads) store_anchor(out + off + q, i, s[q]);
    __syncthreads();
  }
}

// Sorted keys of s[0, n) (n <= kLargeCap): a bitonic network for up to 1024
// keys (padded to a power of two with ~0), the radix sort past that. Returns
// the buffer holding the result (s or t).
__device__ uint64_t* cta_sort_keys(uint64_t* s, uint64_t* t, uint32_t n, uint32_t* whist, uint32_t* dstart,
                                   uint32_t* warp_buf) {
  if (n <= 1024) {
    uint32_t n_pad = 1;
    while (n_pad < n) n_pad <<= 1;
    for (uint32_t q = n + threadIdx.x; q < n_pad; q += blockDim.x) s[q] = ~0ULL;
    __syncthreads();
    bitonic_sort_smem(s, n_pad);
    return s;
  }
  int lb, hb;
  key_field_bits(s, n, &lb, &hb, warp_buf);
  return cta_radix_sort(s, t, n, lb, hb, whist, dstart, warp_buf);
}

// Stable CTA radix sort of a[0, n) (n <= kLargeCap) by the digits of bits
// [0, lo_bits) and [32, 32 + hi_bits), 8 bits at a time (the anchor key's
// read-position field and its reference-position field; bits outside them are
// zero in every key). Warp w ranks the contiguous block of elements
// [w C, w C + C) round by round: the lanes with an equal digit come from
// ballots over the digit's bits, their count from a per-warp counter. Returns
// the buffer (a or b) that holds the result.
__device__ uint64_t* cta_radix_sort(uint64_t* a, uint64_t* b, uint32_t n, int lo_bits, int hi_bits,
                                    uint32_t* whist, uint32_t* dstart, uint32_t* warp_buf) {
  constexpr int W = kLargeThreads / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t C = ((n + W * 32 - 1) / (W * 32)) * 32;   // elements per warp, a multiple of 32
  const uint32_t w0 = wid * C, w1 = min(n, w0 + C);
  for (int range = 0; range < 2; ++range) {
    const int base = range ? 32 : 0, bits = range ? hi_bits : lo_bits;
    for (int sh = 0; sh < bits; sh += 8) {
      const int nb = min(8, bits - sh), shift = base + sh;
      const uint32_t dmask = (1u << nb) - 1u;
      for (int i = threadIdx.x; i < W * 256; i += kLargeThreads) whist[i] = 0;
      __syncthreads();
      uint32_t rank[kLargeRounds];
      uint32_t* wh = whist + wid * 256;
      const int rounds = (int)(C / 32);   // the same for every warp
#pragma unroll
      for (int r = 0; r < kLargeRounds; ++r) {
        if (r >= rounds) break;
        const uint32_t idx = w0 + r * 32 + lane;
        const bool ok = idx < w1;
        const uint32_t d = ok ? (uint32_t)(a[idx] >> shift) & dmask : 0u;
        unsigned peers = __ballot_sync(0xffffffffu, ok);
        for (int t = 0; t < nb; ++t) {
          const bool one = (d >> t) & 1u;
          const unsigned bal = __ballot_sync(0xffffffffu, one);
          peers &= one ? bal : ~bal;
        }
        const uint32_t before = ok ? wh[d] : 0u;
        __syncwarp();
        if (ok && (peers & lt) == 0) wh[d] = before + __popc(peers);
        __syncwarp();
        rank[r] = before + __popc(peers & lt);
      }
      __syncthreads();
      uint32_t cnt = 0;
      if (threadIdx.x < 256) {
        for (int w = 0; w < W; ++w) {
          const uint32_t x = whist[w * 256 + threadIdx.x];
          whist[w * 256 + threadIdx.x] = cnt;
          cnt += x;
        }
      }
      uint32_t tot;
      const uint32_t ds = block_excl_scan_u32(cnt, &tot, warp_buf);
      if (threadIdx.x < 256) dstart[threadIdx.x] = ds;
      __syncthreads();
#pragma unroll
      for (int r = 0; r < kLargeRounds; ++r) {
        if (r >= rounds) break;
        const uint32_t idx = w0 + r * 32 + lane;
        if (idx < w1) {
          const uint64_t key = a[idx];
          const uint32_t d = (uint32_t)(key >> shift) & dmask;
          b[dstart[d] + whist[wid * 256 + d] + rank[r]] = key;
        }
      }
      __syncthreads();
      uint64_t* t = a;
      a = b;
      b = t;
    }
  }
  return a;
}

// Bits needed by the read-position field (bits 0..31) and the reference
// position field (bits 32..63) of the keys s[0, n) (block-wide maxima).
__device__ void key_field_bits(const uint64_t* s, uint32_t n, int* lo_bits, int* hi_bits, uint32_t* warp_buf) {
  if (threadIdx.x == 0) {
    warp_buf[0] = 0;
    warp_buf[1] = 0;
  }
  __syncthreads();
  uint32_t lo = 0, hi = 0;
  for (uint32_t q = threadIdx.x; q < n; q += blockDim.x) {
    lo |= (uint32_t)s[q];
    hi |= (uint32_t)(s[q] >> 32);
  }
  lo = __reduce_or_sync(0xffffffffu, lo);
  hi = __reduce_or_sync(0xffffffffu, hi);
  if ((threadIdx.x & 31) == 0) {
    atomicOr(&warp_buf[0], lo);
    atomicOr(&warp_buf[1], hi);
  }
  __syncthreads();
  *lo_bits = 32 - __clz(warp_buf[0]);
  *hi_bits = 32 - __clz(warp_buf[1]);
  __syncthreads();
}

// CTAs take work from a shared counter: first the kLargeCap-anchor chunks of
// the huge reads (each filled, sorted and written to its read's first merge
// buffer in tmp, at twice the read's anchor offset), then the large reads
// (filled, sorted and stored whole). Spreading a huge read's chunks over CTAs
// matters: sorted by one CTA, a 90 kb read with 24,000 anchors held the whole
// launch on one SM while the others idled (71 % of SM cycles idle).
__global__ void __launch_bounds__(kLargeThreads) fill_sort_large(RecSets sets, const uint32_t* __restrict__ src,
                                                                 const uint32_t* __restrict__ seed_seg,
                                                                 const uint64_t* __restrict__ read_off,
                                                                 const uint32_t* __restrict__ huge,
                                                                 const uint64_t* __restrict__ tasks, uint32_t n_tasks,
                                                                 const uint32_t* __restrict__ large, uint32_t n_large,
                                                                 const uint64_t* __restrict__ ent,
                                                                 god_anchor* __restrict__ out, uint64_t* tmp,
                                                                 unsigned int* queue) {
  extern __shared__ __align__(16) uint64_t sk[];  // two buffers of kLargeCap keys, then radix counters
  uint64_t* sb = sk + kLargeCap;
  uint32_t* whist = reinterpret_cast<uint32_t*>(sb + kLargeCap);
  uint32_t* dstart = whist + (kLargeThreads / 32) * 256;
  __shared__ uint32_t warp_buf[kLargeThreads / 32 + 1];
  __shared__ uint32_t s_li;
  const uint32_t nl = n_tasks + n_large;
  while (true) {
    if (threadIdx.x == 0) s_li = atomicAdd(queue, 1u);
    __syncthreads();
    const uint32_t li = s_li;
    __syncthreads();
    if (li >= nl) break;
    const bool chunk = li < n_tasks;
    const uint64_t task = chunk ? tasks[li] : 0;
    const uint32_t i = chunk ? huge[task >> 32] : large[li - n_tasks];
    const uint64_t off = read_off[i];
    const uint64_t n = read_off[i + 1] - off;
    const RecSet S = pick_set(sets, src[i]);
    const uint32_t g = seed_seg[i];
    const uint64_t beg = S.seg_off[g];
    const uint32_t cnt = S.seg_cnt[g];
    const uint64_t c0 = chunk ? (task & 0xFFFFFFFFull) * kLargeCap : 0;
    const uint32_t m = (uint32_t)std::min<uint64_t>(n - c0, kLargeCap);
    fill_range(S, beg, cnt, ent, c0, c0 + m, sk, warp_buf);
    __syncthreads();
    const uint64_t* srt = cta_sort_keys(sk, sb, m, whist, dstart, warp_buf);
    if (chunk) {
      uint64_t* t0 = tmp + 2 * off;
      for (uint32_t q = threadIdx.x; q < m; q += blockDim.x) t0[c0 + q] = srt[q];
    } else {
      for (uint32_t q = threadIdx.x; q < m; q += blockDim.x) store_anchor(out + off + q, i, srt[q]);
    }
    __syncthreads();
  }
}

// Merge levels of the huge reads: level L (1, 2, ...) merges pairs of sorted
// runs of kLargeCap << (L - 1) keys from one of the read's two buffers in tmp
// into the other; a read whose chunks are all merged at this level writes its
// anchors out instead. One CTA per output tile of kLargeCap keys (tiles never
// straddle a pair); each thread finds its start on the merge path by a binary
// search and merges kMergeIpt keys.
constexpr int kMergeIpt = 8;
__global__ void __launch_bounds__(kLargeThreads) merge_huge_level(const uint32_t* __restrict__ huge,
                                                                  const uint64_t* __restrict__ tasks, uint32_t n_tasks,
                                                                  const uint64_t* __restrict__ read_off, uint64_t* tmp,
                                                                  int level, god_anchor* __restrict__ out) {
  const uint64_t R = (uint64_t)kLargeCap << (level - 1);
  for (uint32_t t = blockIdx.x; t < n_tasks; t += gridDim.x) {
    const uint64_t task = tasks[t];
    const uint32_t i = huge[task >> 32];
    const uint64_t off = read_off[i];
    const uint64_t n = read_off[i + 1] - off;
    if (n <= R) continue;                                    // finished at an earlier level
    const bool last = n <= 2 * R;
    const uint64_t* A = tmp + 2 * off + ((level - 1) & 1 ? n : 0);
    uint64_t* D = tmp + 2 * off + ((level - 1) & 1 ? 0 : n);
    const uint64_t t0 = (task & 0xFFFFFFFFull) * kLargeCap;  // first output of the tile
    const uint64_t j = t0 / (2 * R) * (2 * R);               // its pair
    const uint64_t na = std::min<uint64_t>(R, n - j);
    const uint64_t nb = j + R < n ? std::min<uint64_t>(R, n - j - R) : 0;
    const uint64_t* a = A + j;
    const uint64_t* b = a + na;
    const uint64_t d_end = std::min<uint64_t>(t0 - j + kLargeCap, na + nb);
    for (uint64_t d0 = t0 - j + (uint64_t)threadIdx.x * kMergeIpt; d0 < d_end;
         d0 += (uint64_t)blockDim.x * kMergeIpt) {
      uint64_t lo = d0 > nb ? d0 - nb : 0, hi = d0 < na ? d0 : na;
      while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid] <= b[d0 - 1 - mid]) lo = mid + 1; else hi = mid;
      }
      uint64_t x = lo, y = d0 - lo;
      for (int u = 0; u < kMergeIpt && d0 + u < d_end; ++u) {
        const uint64_t key = (y >= nb || (x < na && a[x] <= b[y])) ? a[x++] : b[y++];
        if (last) store_anchor(out + off + j + d0 + u, i, key);
        else D[j + d0 + u] = key;
      }
    }
  }
}

// Looks up U records (rp[u] valid when ok[u]) and writes (read position << 1
// | z) and the lookup result (start | count << 32) to pz / sc at oi[u].
template <int VIA, int U>
__device__ __forceinline__ void lookup_records(const RmiRoot& R, const DeviceIndex& di, const MinRec* const (&rp)[U],
                                               const bool (&ok)[U], const uint64_t (&oi)[U],
                                               uint32_t* __restrict__ pz, uint64_t* __restrict__ sc) {
  uint64_t key[U], rk[U];
  uint32_t pzv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    uint4 r = make_uint4(0, 0, 0, 0);
    if (ok[u]) r = __ldcs(reinterpret_cast<const uint4*>(rp[u]));   // read once
    key[u] = ((uint64_t)r.y << 32) | r.x;
    pzv[u] = (r.z << 1) | (r.w & 1u);
  }
  uint64_t pay[U];
  if (VIA == 1) {
    RmiLeaf L[U];
    bool hashed[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      hashed[u] = !rmi_in_range(R, key[u]);
      L[u] = ok[u] && !hashed[u] ? di.leaves[rmi_root_leaf(R, key[u])] : RmiLeaf{0, 0.0f, 0.0f};
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      hashed[u] = hashed[u] || (uint32_t)(L[u].base_eps >> 56) > di.eps_max;
      pay[u] = !ok[u] ? 0 : hashed[u] ? ht_find(di, key[u]) : rank_payload(di, rmi_rank_in_leaf(di, L[u], key[u]));
    }
  } else {
    uint64_t w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) w[u] = ok[u] ? ht_home_word(di, key[u]) : kEmptyKey;
#pragma unroll
    for (int u = 0; u < U; ++u) rk[u] = ok[u] ? ht_field(di, key[u], w[u]) : kNoRank;
#pragma unroll
    for (int u = 0; u < U; ++u) pay[u] = field_payload(di, rk[u]);
  }
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (ok[u]) {
      pz[oi[u]] = pzv[u];
      sc[oi[u]] = pay[u];
    }
  }
}

// Staged sketch output (tile kernel: WT slots per warp sub-tile) -> ordered
// per-record (position << 1 | z) words and index lookups, a warp per
// sub-tile. The key is not kept: nothing after the lookup needs it.
template <int VIA>
__global__ void __launch_bounds__(kT) compact_lookup(const MinRec* __restrict__ staging,
                                                     const uint32_t* __restrict__ sub_cnt,
                                                     const uint64_t* __restrict__ sub_off, uint64_t n_sub, int WT,
                                                     DeviceIndex di, uint32_t* __restrict__ pz,
                                                     uint64_t* __restrict__ sc) {
  __shared__ RmiRoot R;
  if (VIA == 1) {
    if (threadIdx.x == 0) R = *di.root;
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t sub = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; sub < n_sub; sub += warps) {
    const uint32_t c = sub_cnt[sub];
    const uint64_t o = sub_off[sub];
    const MinRec* src = staging + sub * (uint64_t)WT;
    // two records per lane, each dependent step issued for both first (more in
    // flight per lane measured slower)
    constexpr int U = 2;
    for (uint32_t i0 = lane; i0 < c; i0 += 32 * U) {
      const MinRec* rp[U];
      bool ok[U];
      uint64_t oi[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = i0 + 32 * u;
        ok[u] = i < c;
        rp[u] = src + i;
        oi[u] = o + i;
      }
      lookup_records<VIA, U>(R, di, rp, ok, oi, pz, sc);
    }
  }
}

// The same for the per-segment kernel's staging (segment s's records at
// staging[base[s]]): a warp takes 32 consecutive segments and spreads their
// records over its lanes; a lane finds the segment of its record by a binary
// search over the segments' exclusive counts held one per lane.
template <int VIA>
__global__ void __launch_bounds__(kT) compact_lookup_seg(const MinRec* __restrict__ staging,
                                                         const uint32_t* __restrict__ sub_cnt,
                                                         const uint64_t* __restrict__ sub_off, uint64_t n_sub,
                                                         const uint64_t* __restrict__ base, DeviceIndex di,
                                                         uint32_t* __restrict__ pz, uint64_t* __restrict__ sc) {
  __shared__ RmiRoot R;
  if (VIA == 1) {
    if (threadIdx.x == 0) R = *di.root;
    __syncthreads();
  }
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t grp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; grp * 32 < n_sub; grp += warps) {
    const uint64_t s = grp * 32 + lane;
    const uint32_t c = s < n_sub ? sub_cnt[s] : 0u;
    const uint64_t b = s < n_sub ? base[s] : 0;
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, d);
      if (lane >= d) inc += y;
    }
    const uint32_t ex = inc - c;
    const uint32_t tot = __shfl_sync(FULL, inc, 31);
    const uint64_t o0 = sub_off[grp * 32];
    constexpr int U = 2;
    // warp-uniform trip count: every lane takes part in the shuffles
    for (uint32_t b0 = 0; b0 < tot; b0 += 32 * U) {
      const MinRec* rp[U];
      bool ok[U];
      uint64_t oi[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const uint32_t i = b0 + lane + 32 * u;
        ok[u] = i < tot;
        int L = 0;   // last lane whose segment starts at or before record i
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t e = __shfl_sync(FULL, ex, L + step);
          if (e <= i) L += step;
        }
        const uint32_t eL = __shfl_sync(FULL, ex, L);
        const uint64_t bL = __shfl_sync(FULL, b, L);
        rp[u] = staging + bL + (i - eL);
        oi[u] = o0 + i;
      }
      lookup_records<VIA, U>(R, di, rp, ok, oi, pz, sc);
    }
  }
}

// One record set: sketch + lookup + per-segment offsets.
struct SetBufs {
  DBuf<SegDesc> segs;
  DBuf<uint32_t> vlen;
  DBuf<uint64_t> voff;
  DBuf<uint32_t> pz;
  DBuf<uint64_t> sc;
  DBuf<uint32_t> seg_cnt;
  DBuf<uint64_t> seg_off;
  DBuf<uint32_t> max_m;      // longest segment (set by the segment builders)
  uint32_t max_m_host = 0;   // its value, read back with the stream length
  uint64_t n_seg = 0;
  RecSet view() const { return RecSet{pz.p, sc.p, seg_off.p, seg_cnt.p}; }
};

// err (optional, device int) is read back together with the stream length;
// a non-zero value means the offsets were invalid.
int sketch_and_lookup(const god_index* idx, const uint8_t* d_reads, SetBufs& B, uint32_t* read_flag, int via,
                      const int* err, cudaStream_t st) {
  GOD_TRY(B.voff.alloc(B.n_seg + 1, st));
  GOD_TRY(exclusive_scan_u32(B.vlen.p, B.voff.p, B.n_seg, st));
  uint64_t V = 0;
  int herr = 0;
  uint32_t max_m = 0;
  GOD_CK(cudaMemcpyAsync(&V, B.voff.p + B.n_seg, 8, cudaMemcpyDeviceToHost, st));
  if (err) GOD_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (B.max_m.p) GOD_CK(cudaMemcpyAsync(&max_m, B.max_m.p, 4, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  if (herr) {
    set_error("seed: offsets must be non-decreasing and each read < 2^31 bytes");
    return GOD_EINVAL;
  }
  GOD_TRY(scan_total_ok(V, "seed"));
  GOD_TRY(B.seg_cnt.alloc(B.n_seg, st));
  SketchJob job{};
  job.bytes = d_reads;
  job.segs = B.segs.p;
  job.seg_voff = B.voff.p;
  job.n_seg = (uint32_t)B.n_seg;
  job.V = V;
  job.k = idx->k;
  job.w = idx->w;
  job.pat = idx->pat;
  job.seg_cnt = B.seg_cnt.p;
  job.read_flag = read_flag;
  job.tune = idx->params.tune;
  job.max_m = max_m;
  B.max_m_host = max_m;
  job.bytes_on_host = is_device_ptr(d_reads) ? 0 : 1;
  const DeviceIndex di = device_view(idx, via);
  const bool learned = via == 1 && di.leaves;
  StagedSketch SS;
  if (V > 0 && sketch_segments_ok(job)) {
    // short segments, one thread each: the record total stays on the device
    // (pz / sc sized for V records, its bound), and the segment offsets are
    // the pass's own sub-tile offsets
    GOD_TRY(run_sketch_segments(job, st, SS));
    GOD_TRY(B.pz.alloc(V, st));
    GOD_TRY(B.sc.alloc(V, st));
    const unsigned blocks =
        (unsigned)std::min<uint64_t>(((SS.n_sub + 31) / 32 * 32 + kT - 1) / kT, (uint64_t)num_sms() * 16);
    if (learned)
      GOD_LAUNCH(compact_lookup_seg<1>, blocks, kT, 0, st, SS.staging.p, SS.sub_cnt.p, SS.sub_off.p, SS.n_sub,
                 SS.sub_base, di, B.pz.p, B.sc.p);
    else
      GOD_LAUNCH(compact_lookup_seg<0>, blocks, kT, 0, st, SS.staging.p, SS.sub_cnt.p, SS.sub_off.p, SS.n_sub,
                 SS.sub_base, di, B.pz.p, B.sc.p);
    // algorithmic bytes: record read 16, position word 4, result 8, one table
    // slot 8 and the key's two offsets 8
    prof_add_work_async(learned ? "compact_lookup_seg<1>" : "compact_lookup_seg<0>",
                        reinterpret_cast<const unsigned long long*>(SS.sub_off.p + SS.n_sub), 0.0, 44.0, 0.0, 1.0,
                        st);
    B.seg_off.st = st;
    B.seg_off.n = SS.sub_off.n;
    B.seg_off.p = SS.sub_off.take();
    return GOD_OK;
  }
  GOD_TRY(run_sketch_staged(job, st, SS, nullptr));
  GOD_TRY(B.pz.alloc(SS.total, st));
  GOD_TRY(B.sc.alloc(SS.total, st));
  if (SS.total) {
    const unsigned blocks = (unsigned)std::min<uint64_t>((SS.n_sub * 32 + kT - 1) / kT, (uint64_t)num_sms() * 16);
    if (learned)
      GOD_LAUNCH(compact_lookup<1>, blocks, kT, 0, st, SS.staging.p, SS.sub_cnt.p, SS.sub_off.p, SS.n_sub, SS.WT, di,
                 B.pz.p, B.sc.p);
    else
      GOD_LAUNCH(compact_lookup<0>, blocks, kT, 0, st, SS.staging.p, SS.sub_cnt.p, SS.sub_off.p, SS.n_sub, SS.WT, di,
                 B.pz.p, B.sc.p);
    // algorithmic bytes: record read 16, position word 4, result 8, one table
    // slot 8 and the key's two offsets 8
    prof_add_work(learned ? "compact_lookup<1>" : "compact_lookup<0>", 44.0 * (double)SS.total, (double)SS.total);
  }
  GOD_TRY(B.seg_off.alloc(B.n_seg + 1, st));
  GOD_TRY(exclusive_scan_u32(B.seg_cnt.p, B.seg_off.p, B.n_seg, st));
  return GOD_OK;
}

}  // namespace

int seed_device(const god_index* idx, const uint8_t* d_reads, const uint64_t* d_offs, uint32_t n, uint64_t read_bytes,
                const god_seed_opts& o, cudaStream_t st, god_anchor** d_out, uint64_t* n_anchors, god_anchor* user_out,
                uint64_t user_cap, bool user_out_device) {
  (void)read_bytes;
  (void)user_out_device;
  *n_anchors = 0;
  if (n == 0) return GOD_OK;
  const PatternInfo& P = idx->pat;
  const int p = P.p;
  const uint32_t t = (o.pa_t != UINT32_MAX) ? o.pa_t : idx->params.pa_t;
  const int via = (o.via < 0) ? (idx->params.index_kind == GOD_INDEX_LEARNED && idx->has_rmi ? 1 : 0)
                              : ((o.via == 1 && idx->has_rmi) ? 1 : 0);
  const int k = idx->k, w = idx->w;
  if ((uint64_t)n * p >= (1ull << 31)) {
    set_error("seed: too many reads for this pattern length");
    return GOD_EINVAL;
  }
  // prefix cap for pattern alignment (odd k only: even k admits palindromic
  // windows without a minimizer, which would void the prefix guarantee)
  uint32_t cap = 0xFFFFFFFEu;
  if (t > 0 && (k & 1)) {
    const uint64_t c = (uint64_t)t * w + w + k - 2;
    if (c < cap) cap = (uint32_t)c;
  }

  // small per-call state: error flag, list counters and work queues in one buffer
  constexpr int kCtl = 13;
  DBuf<unsigned long long> ctl;
  GOD_TRY(ctl.alloc(kCtl, st));
  GOD_CK(cudaMemsetAsync(ctl.p, 0, kCtl * sizeof(unsigned long long), st));
  int* err = reinterpret_cast<int*>(ctl.p);
  unsigned long long* pa_counts = ctl.p + 1;     // [fallback, seeding pass]
  // [tiny, small, warp, medium, large, huge, huge chunks, most chunks]
  unsigned long long* fill_counts = ctl.p + 3;
  unsigned int* fill_queue = reinterpret_cast<unsigned int*>(ctl.p + 11);
  unsigned long long* task_ctr = ctl.p + 12;
  DBuf<uint32_t> need_full, shift, src, seed_seg, fb_list, p2_list;
  DBuf<uint64_t> read_cnt, read_off;
  GOD_TRY(need_full.alloc(n, st));
  GOD_TRY(shift.alloc(n, st));
  GOD_TRY(src.alloc(n, st));
  GOD_TRY(seed_seg.alloc(n, st));
  GOD_TRY(fb_list.alloc(n, st));
  GOD_TRY(p2_list.alloc(n, st));
  GOD_TRY(read_cnt.alloc(n, st));
  GOD_TRY(read_off.alloc((uint64_t)n + 1, st));
  GOD_CK(cudaMemsetAsync(need_full.p, 0, n * sizeof(uint32_t), st));

  // ---- PA pass
  SetBufs PA;
  PA.n_seg = (uint64_t)n * p;
  GOD_TRY(PA.segs.alloc(PA.n_seg, st));
  GOD_TRY(PA.vlen.alloc(PA.n_seg, st));
  GOD_TRY(PA.max_m.alloc(1, st));
  GOD_CK(cudaMemsetAsync(PA.max_m.p, 0, 4, st));
  GOD_LAUNCH(make_pa_segments, grid_for(n), kT, 0, st, d_offs, n, P, cap, PA.segs.p, PA.vlen.p, err, PA.max_m.p);
  GOD_TRY(sketch_and_lookup(idx, d_reads, PA, need_full.p, via, err, st));
  GOD_LAUNCH(pa_select, grid_for(n), kT, 0, st, n, p, t, PA.segs.p, PA.view(), need_full.p, shift.p, src.p,
             seed_seg.p, read_cnt.p, fb_list.p, p2_list.p, pa_counts);
  unsigned long long hc[2] = {0, 0};
  uint64_t pa_tot = 0;
  // Both follow-up passes come from segments cut at the cap (a fallback for an
  // N in a cut prefix, a seeding pass for a read whose chosen prefix was cut):
  // when every segment is shorter than the cap there are none, and the counts
  // need not be read back here (the record total is checked with the others).
  const bool cut = PA.max_m_host >= cap;
  if (cut) {
    GOD_CK(cudaMemcpyAsync(hc, pa_counts, sizeof(hc), cudaMemcpyDeviceToHost, st));
    GOD_CK(cudaMemcpyAsync(&pa_tot, PA.seg_off.p + PA.n_seg, 8, cudaMemcpyDeviceToHost, st));
    GOD_CK(cudaStreamSynchronize(st));
    GOD_TRY(scan_total_ok(pa_tot, "seed"));
  }
  const uint64_t n_fb = hc[0], n_p2 = hc[1];

  // ---- fallback: full-length pattern alignment for reads with N in the prefix
  SetBufs FB;
  if (n_fb) {
    FB.n_seg = n_fb * p;
    GOD_TRY(FB.segs.alloc(FB.n_seg, st));
    GOD_TRY(FB.vlen.alloc(FB.n_seg, st));
    GOD_TRY(FB.max_m.alloc(1, st));
    GOD_CK(cudaMemsetAsync(FB.max_m.p, 0, 4, st));
    GOD_LAUNCH(make_list_segments, grid_for(n_fb), kT, 0, st, d_offs, fb_list.p, (uint32_t)n_fb, P, 1, shift.p,
               FB.segs.p, FB.vlen.p, FB.max_m.p);
    GOD_TRY(sketch_and_lookup(idx, d_reads, FB, nullptr, via, nullptr, st));
    GOD_LAUNCH(pa_select_list, grid_for(n_fb), kT, 0, st, fb_list.p, (uint32_t)n_fb, p, t, FB.view(), shift.p,
               seed_seg.p, read_cnt.p);
  }
  // ---- seeding pass for reads whose shift-a segment was a prefix
  SetBufs P2;
  if (n_p2) {
    P2.n_seg = n_p2;
    GOD_TRY(P2.segs.alloc(P2.n_seg, st));
    GOD_TRY(P2.vlen.alloc(P2.n_seg, st));
    GOD_TRY(P2.max_m.alloc(1, st));
    GOD_CK(cudaMemsetAsync(P2.max_m.p, 0, 4, st));
    GOD_LAUNCH(make_list_segments, grid_for(n_p2), kT, 0, st, d_offs, p2_list.p, (uint32_t)n_p2, P, 0, shift.p,
               P2.segs.p, P2.vlen.p, P2.max_m.p);
    GOD_TRY(sketch_and_lookup(idx, d_reads, P2, nullptr, via, nullptr, st));
    GOD_LAUNCH(set_seed_seg_list, grid_for(n_p2), kT, 0, st, p2_list.p, (uint32_t)n_p2, seed_seg.p);
    GOD_LAUNCH(count_anchors_list, grid_for(n_p2 * 32), kT, 0, st, p2_list.p, (uint32_t)n_p2, P2.view(),
               read_cnt.p);
  }
  if (o.shifts_out) {
    GOD_CK(cudaMemcpyAsync(o.shifts_out, shift.p, n * sizeof(uint32_t), cudaMemcpyDefault, st));
  }

  // ---- anchors per read: offsets, length classes
  RecSets sets;
  sets.s[kSrcPA] = PA.view();
  sets.s[kSrcFB] = FB.view();
  sets.s[kSrcP2] = P2.view();
  GOD_TRY(exclusive_scan_u64(read_cnt.p, read_off.p, n, st));
  DBuf<uint32_t> ltiny, lsmall, lwarp, lmedium, llarge, lhuge;
  GOD_TRY(ltiny.alloc(n, st));
  GOD_TRY(lsmall.alloc(n, st));
  GOD_TRY(lwarp.alloc(n, st));
  GOD_TRY(lmedium.alloc(n, st));
  GOD_TRY(llarge.alloc(n, st));
  GOD_TRY(lhuge.alloc(n, st));
  GOD_LAUNCH(classify_reads, grid_for(n), kT, 0, st, n, read_off.p, ltiny.p, lsmall.p, lwarp.p, lmedium.p,
             llarge.p, lhuge.p, fill_counts);
  uint64_t total = 0;
  unsigned long long hf[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  uint64_t set_tot[2] = {0, 0};
  GOD_CK(cudaMemcpyAsync(&total, read_off.p + n, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaMemcpyAsync(hf, fill_counts, sizeof(hf), cudaMemcpyDeviceToHost, st));
  if (!cut) GOD_CK(cudaMemcpyAsync(&pa_tot, PA.seg_off.p + PA.n_seg, 8, cudaMemcpyDeviceToHost, st));
  if (n_fb) GOD_CK(cudaMemcpyAsync(&set_tot[0], FB.seg_off.p + FB.n_seg, 8, cudaMemcpyDeviceToHost, st));
  if (n_p2) GOD_CK(cudaMemcpyAsync(&set_tot[1], P2.seg_off.p + P2.n_seg, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  GOD_TRY(scan_total_ok(pa_tot, "seed"));
  GOD_TRY(scan_total_ok(total, "seed"));
  GOD_TRY(scan_total_ok(set_tot[0], "seed"));
  GOD_TRY(scan_total_ok(set_tot[1], "seed"));
  *n_anchors = total;
  god_anchor* out = user_out;
  if (user_out) {
    if (total > user_cap) return GOD_ERANGE;
  } else {
    GOD_TRY(dmalloc((void**)&out, std::max<uint64_t>(total, 1) * sizeof(god_anchor), st));
    *d_out = out;
  }
  if (total == 0) return GOD_OK;

  // ---- fill + sort per read
  const uint64_t n_tiny = hf[0], n_small = hf[1], n_warp = hf[2], n_medium = hf[3], n_large = hf[4],
                 n_huge = hf[5];
  if (n_tiny)
    GOD_LAUNCH(fill_sort_tiny, grid_for(n_tiny, kT, 64), kT, 0, st, sets, src.p, seed_seg.p, read_off.p, ltiny.p,
               (uint32_t)n_tiny, idx->d_ent, out);
  if (n_small)
    GOD_LAUNCH(fill_sort_small, grid_for(n_small * 32, kT, 64), kT, 0, st, sets, src.p, seed_seg.p, read_off.p,
               lsmall.p, (uint32_t)n_small, idx->d_ent, out);
  if (n_warp)
    GOD_LAUNCH(fill_sort_warp, grid_for(n_warp * 32, kT, 64), kT, 0, st, sets, src.p, seed_seg.p, read_off.p, lwarp.p,
               (uint32_t)n_warp, idx->d_ent, out);
  if (n_medium)
    GOD_LAUNCH(fill_sort_medium, (unsigned)std::min<uint64_t>(n_medium, (uint64_t)num_sms() * 16), kMedThreads, 0,
               st, sets, src.p, seed_seg.p, read_off.p, lmedium.p, (uint32_t)n_medium, idx->d_ent, out);
  if (n_large + n_huge) {
    // huge reads: one task per kLargeCap-anchor tile, two merge buffers per
    // read in tmp (at twice its anchor offset), ceil(log2(most tiles)) levels
    const uint64_t n_tasks = hf[6], most = hf[7];
    if (n_tasks >= (1ull << 31)) {
      set_error("seed: too many long anchor lists in one call");
      return GOD_ERANGE;
    }
    DBuf<uint64_t> tmp, tasks;
    if (n_huge) {
      GOD_TRY(tmp.alloc(2 * total, st));
      GOD_TRY(tasks.alloc(n_tasks, st));
      GOD_LAUNCH(huge_tasks, grid_for(n_huge), kT, 0, st, lhuge.p, (uint32_t)n_huge, read_off.p, tasks.p, task_ctr);
    }
    const size_t smem = 2 * kLargeCap * sizeof(uint64_t) + (kLargeThreads / 32) * 256 * 4 + 256 * 4;
    GOD_CK(cudaFuncSetAttribute(fill_sort_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)std::min<uint64_t>(n_large + n_tasks, (uint64_t)num_sms() * 3);
    GOD_LAUNCH(fill_sort_large, grid, kLargeThreads, smem, st, sets, src.p, seed_seg.p, read_off.p, lhuge.p, tasks.p,
               (uint32_t)n_tasks, llarge.p, (uint32_t)n_large, idx->d_ent, out, tmp.p, fill_queue);
    int levels = 0;
    while ((1ull << levels) < most) ++levels;
    const unsigned mgrid = (unsigned)std::min<uint64_t>(std::max<uint64_t>(n_tasks, 1), (uint64_t)num_sms() * 8);
    for (int L = 1; L <= levels; ++L)
      GOD_LAUNCH(merge_huge_level, mgrid, kLargeThreads, 0, st, lhuge.p, tasks.p, (uint32_t)n_tasks, read_off.p, tmp.p,
                 L, out);
  }
  return GOD_OK;
}

}  // namespace god
