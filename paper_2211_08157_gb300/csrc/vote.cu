// Location voting on each read's anchors (Sec. 3.4 steps 1-5, Fig. 8) with the
// rescue location (Sec. 3.6.3).
//
// Per read:
//  1. every anchor becomes one vote at a signed location: v = ref_pos -
//     read_pos on the forward strand, v = ref_pos - (len - 1 - read_pos) on the
//     reverse strand (the read position counted from the read's other end);
//  2. the votes are sorted by (strand, v): the 64-bit sort key is
//     strand << 63 | (v + 2^32) << 28 | i, with i the anchor's index inside
//     the read's list (unique keys; the index also leads back to the anchor's
//     positions);
//  3-5. one warp walks the sorted votes 32 at a time: a group opens at the
//     first vote left, takes every vote of its strand within D of it (a
//     contiguous run of lanes, found by one ballot), and closes at the first
//     vote beyond; closed groups with at least V votes enter a top list kept
//     one entry per lane (votes descending, discovery order on ties, cut at
//     max_out), and the group with the most votes is kept as the rescue.
// Lists of up to 16 votes are sorted in one thread's registers and walked by
// that thread (when at most 8 winners are kept); up to 32 by a warp (bitonic
// network over shuffles, then the warp's walk); longer ones by a CTA in shared memory (bitonic network up to
// 4096 keys), and lists past 4096 in sorted chunks merged by merge-path
// passes in a global buffer. CTAs take long reads from a shared counter,
// chunked ones first.
#include <algorithm>

#include "common.cuh"

namespace god {
namespace {

constexpr int kVT = 256;                 // threads of the CTA path
constexpr uint32_t kVoteThreadCap = 16;  // votes sorted in one thread's registers
constexpr uint32_t kThreadTop = 8;       // winners a thread keeps (max_out <= 8 for the thread path)
constexpr uint32_t kVoteWarpCap = 32;    // votes sorted in registers by one warp
constexpr uint32_t kVoteCap = 4096;      // votes sorted in shared memory at once
constexpr int kIdxBits = 28;             // anchor index field of the sort key
constexpr uint64_t kIdxMask = (1ull << kIdxBits) - 1;
constexpr uint64_t kVMask = (1ull << 35) - 1;   // v + 2^32 field
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint64_t vote_key(const god_anchor& a, uint64_t len, uint32_t i) {
  const int64_t v = a.strand == 0 ? (int64_t)a.ref_pos - (int64_t)a.read_pos
                                  : (int64_t)a.ref_pos - ((int64_t)len - 1 - (int64_t)a.read_pos);
  return ((uint64_t)(a.strand & 1u) << 63) | (((uint64_t)(v + (1ll << 32)) & kVMask) << kIdxBits) | (uint64_t)i;
}
__device__ __forceinline__ uint32_t key_strand(uint64_t k) { return (uint32_t)(k >> 63); }
__device__ __forceinline__ int64_t key_v(uint64_t k) { return (int64_t)((k >> kIdxBits) & kVMask) - (1ll << 32); }

// Read r's anchors are [read_off[r], read_off[r + 1]): the first index whose
// read id is >= r. err = 1 when the list is not grouped by ascending read id
// or names a read >= n.
__global__ void vote_ranges(const god_anchor* __restrict__ a, uint64_t m, uint32_t n, uint64_t* __restrict__ read_off,
                            int* err) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t cur = i < m ? (uint64_t)a[i].read_id : (uint64_t)n;
    const uint64_t prev = i > 0 ? (uint64_t)a[i - 1].read_id : 0;
    if (i < m && (cur >= n || (i > 0 && cur < prev))) {
      atomicExch(err, 1);
      continue;
    }
    // reads (prev, cur] start here (read 0 included at i = 0)
    const uint64_t lo = i > 0 ? prev + 1 : 0;
    for (uint64_t r = lo; r <= cur && r <= n; ++r) read_off[r] = i;
  }
}

__device__ __forceinline__ void warp_push(bool f, uint32_t v, uint32_t* list, unsigned int* counter) {
  const unsigned am = __activemask();
  const unsigned bal = __ballot_sync(am, f);
  if (!bal) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(am) - 1;
  unsigned int base = 0;
  if (lane == leader) base = atomicAdd(counter, (unsigned int)__popc(bal));
  base = __shfl_sync(am, base, leader);
  if (f) list[base + __popc(bal & ((1u << lane) - 1u))] = v;
}

// counts[r] = 0 for reads without anchors; lists of reads by vote count.
// ctl: [0] warp list, [1] long list, [2] chunked list, [3] queue, [4] error,
// [5] thread list (when max_out allows it).
__global__ void vote_classify(uint32_t n, const uint64_t* __restrict__ read_off, uint32_t* __restrict__ counts,
                              uint32_t* __restrict__ lw, uint32_t* __restrict__ ll, uint32_t* __restrict__ lh,
                              uint32_t* __restrict__ lt, uint32_t thread_cap, unsigned int* ctl) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t c = read_off[r + 1] - read_off[r];
    if (c == 0) counts[r] = 0;
    if (c > kIdxMask) atomicExch(reinterpret_cast<int*>(ctl + 4), 2);
    warp_push(c > 0 && c <= thread_cap, (uint32_t)r, lt, ctl + 5);
    warp_push(c > thread_cap && c <= kVoteWarpCap, (uint32_t)r, lw, ctl + 0);
    warp_push(c > kVoteWarpCap && c <= kVoteCap, (uint32_t)r, ll, ctl + 1);
    warp_push(c > kVoteCap && c <= kIdxMask, (uint32_t)r, lh, ctl + 2);
  }
}

struct VoteCfg {
  uint32_t D, V, max_out;
};

// A group's summary (uniform across the warp).
struct Group {
  uint32_t strand, votes, ref_lo, ref_hi, read_lo, read_hi;
  int64_t v0;
};

// The warp's walk over one read's sorted votes. get(i) returns the i-th key
// (i < n) and the anchor it came from; every lane calls it for its own i.
template <typename Get>
__device__ void vote_walk(uint32_t r, uint32_t n, const VoteCfg& cfg, Get get, god_vote_rec* __restrict__ out,
                          uint32_t* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  // top list: lane j holds entry j (j < cnt)
  Group e{0, 0, 0, 0, 0, 0, 0};
  uint32_t cnt = 0;
  Group best{0, 0, 0, 0, 0, 0, 0};
  bool have_best = false;
  Group g{0, 0, 0, 0, 0, 0, 0};
  bool open = false;
  auto close = [&](const Group& c) {
    if (c.votes >= cfg.V) {
      const bool ge = (uint32_t)lane < cnt && e.votes >= c.votes;
      const uint32_t pos = __popc(__ballot_sync(kFull, ge));
      if (pos < cfg.max_out) {
        Group up;
        up.strand = __shfl_up_sync(kFull, e.strand, 1);
        up.votes = __shfl_up_sync(kFull, e.votes, 1);
        up.ref_lo = __shfl_up_sync(kFull, e.ref_lo, 1);
        up.ref_hi = __shfl_up_sync(kFull, e.ref_hi, 1);
        up.read_lo = __shfl_up_sync(kFull, e.read_lo, 1);
        up.read_hi = __shfl_up_sync(kFull, e.read_hi, 1);
        up.v0 = __shfl_up_sync(kFull, e.v0, 1);
        if ((uint32_t)lane > pos) e = up;
        if ((uint32_t)lane == pos) e = c;
        cnt = min(cnt + 1, cfg.max_out);
      }
    }
    if (!have_best || c.votes > best.votes) {
      best = c;
      have_best = true;
    }
  };
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + lane;
    const bool valid = i < n;
    uint64_t key = ~0ull;
    uint32_t ref = 0, rp = 0;
    if (valid) get(i, &key, &ref, &rp);
    const uint32_t st = key_strand(key);
    const int64_t v = key_v(key);
    const uint32_t here = min(32u, n - base);
    uint32_t pos = 0;
    while (pos < here) {
      if (!open) {
        g.strand = __shfl_sync(kFull, st, pos);
        g.v0 = __shfl_sync(kFull, v, pos);
        g.votes = 0;
        g.ref_lo = 0xffffffffu;
        g.ref_hi = 0;
        g.read_lo = 0xffffffffu;
        g.read_hi = 0;
        open = true;
      }
      const bool in = valid && (uint32_t)lane >= pos && st == g.strand && v - g.v0 <= (int64_t)cfg.D;
      const uint32_t c = __popc(__ballot_sync(kFull, in));
      g.votes += c;
      g.ref_lo = min(g.ref_lo, __reduce_min_sync(kFull, in ? ref : 0xffffffffu));
      g.ref_hi = max(g.ref_hi, __reduce_max_sync(kFull, in ? ref : 0u));
      g.read_lo = min(g.read_lo, __reduce_min_sync(kFull, in ? rp : 0xffffffffu));
      g.read_hi = max(g.read_hi, __reduce_max_sync(kFull, in ? rp : 0u));
      pos += c;
      if (pos < here) {   // the vote at lane pos lies beyond: the group closes
        close(g);
        open = false;
      }
    }
  }
  if (open) close(g);
  const bool rescue = cnt == 0 && have_best;
  const uint32_t total = rescue ? 1u : cnt;
  if ((uint32_t)lane < total) {
    const Group& o = rescue ? best : e;
    god_vote_rec rec;
    rec.read_id = r;
    rec.votes = o.votes;
    rec.strand = o.strand;
    rec.rescue = rescue ? 1u : 0u;
    rec.loc = o.v0;
    rec.ref_lo = o.ref_lo;
    rec.ref_hi = o.ref_hi;
    rec.read_lo = o.read_lo;
    rec.read_hi = o.read_hi;
    out[(uint64_t)r * cfg.max_out + lane] = rec;
  }
  if (lane == 0) counts[r] = total;
}

__device__ __forceinline__ void cswap64(uint64_t& x, uint64_t& y, bool up) {
  const uint64_t lo = x < y ? x : y, hi = x < y ? y : x;
  x = up ? lo : hi;
  y = up ? hi : lo;
}

// Reads with at most 16 votes (and max_out <= 8): a thread per read. The keys
// are sorted by a 16-wide bitonic network in registers, the groups walked in
// order, and the winners kept in a register top list (insertion at the
// number of kept winners with at least as many votes: equal votes keep their
// (strand, v0) order).
constexpr int kVTT = 128;   // threads per block of the thread path (many registers per thread)

__global__ void __launch_bounds__(kVTT) vote_thread(const god_anchor* __restrict__ a,
                                                   const uint64_t* __restrict__ read_off,
                                                   const uint64_t* __restrict__ offs, const uint32_t* __restrict__ list,
                                                   const unsigned int* __restrict__ ctl, VoteCfg cfg,
                                                   god_vote_rec* __restrict__ out, uint32_t* __restrict__ counts) {
  const uint32_t nl = ctl[5];
  for (uint64_t li = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; li < nl; li += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t r = list[li];
    const uint64_t lo = read_off[r];
    const uint32_t n = (uint32_t)(read_off[r + 1] - lo);
    const uint64_t len = offs[r + 1] - offs[r];
    uint64_t kk[kVoteThreadCap];
#pragma unroll
    for (int q = 0; q < (int)kVoteThreadCap; ++q) kk[q] = (uint32_t)q < n ? vote_key(a[lo + q], len, q) : ~0ull;
#pragma unroll
    for (int s2 = 2; s2 <= (int)kVoteThreadCap; s2 <<= 1) {
#pragma unroll
      for (int j = s2 >> 1; j > 0; j >>= 1) {
#pragma unroll
        for (int q = 0; q < (int)kVoteThreadCap; ++q) {
          const int q2 = q ^ j;
          if (q2 > q) cswap64(kk[q], kk[q2], (q & s2) == 0);
        }
      }
    }
    Group e[kThreadTop];
    uint32_t cnt = 0;
    Group best{0, 0, 0, 0, 0, 0, 0};
    Group g{0, 0, 0, 0, 0, 0, 0};
    auto close = [&](const Group& c) {
      if (c.votes >= cfg.V) {
        uint32_t pos = 0;
#pragma unroll
        for (int q = 0; q < (int)kThreadTop; ++q) pos += ((uint32_t)q < cnt && e[q].votes >= c.votes) ? 1u : 0u;
        if (pos < cfg.max_out) {
#pragma unroll
          for (int q = (int)kThreadTop - 1; q > 0; --q)
            if ((uint32_t)q > pos) e[q] = e[q - 1];
#pragma unroll
          for (int q = 0; q < (int)kThreadTop; ++q)
            if ((uint32_t)q == pos) e[q] = c;
          cnt = min(cnt + 1, cfg.max_out);
        }
      }
      if (c.votes > best.votes) best = c;   // groups have >= 1 vote: the first one always enters
    };
#pragma unroll
    for (int q = 0; q < (int)kVoteThreadCap; ++q) {
      if ((uint32_t)q < n) {
        const uint64_t key = kk[q];
        const god_anchor an = a[lo + (key & kIdxMask)];
        const uint32_t st = key_strand(key);
        const int64_t v = key_v(key);
        if (q > 0 && (st != g.strand || v - g.v0 > (int64_t)cfg.D)) close(g);
        if (q == 0 || st != g.strand || v - g.v0 > (int64_t)cfg.D) {
          g.strand = st;
          g.v0 = v;
          g.votes = 0;
          g.ref_lo = g.read_lo = 0xffffffffu;
          g.ref_hi = g.read_hi = 0;
        }
        g.votes++;
        g.ref_lo = min(g.ref_lo, an.ref_pos);
        g.ref_hi = max(g.ref_hi, an.ref_pos);
        g.read_lo = min(g.read_lo, an.read_pos);
        g.read_hi = max(g.read_hi, an.read_pos);
      }
    }
    close(g);
    const bool rescue = cnt == 0;
    const uint32_t total = rescue ? 1u : cnt;
    god_vote_rec* o = out + (uint64_t)r * cfg.max_out;
#pragma unroll
    for (int q = 0; q < (int)kThreadTop; ++q) {
      if ((uint32_t)q < total) {
        const Group& s = rescue ? best : e[q];
        god_vote_rec rec;
        rec.read_id = r;
        rec.votes = s.votes;
        rec.strand = s.strand;
        rec.rescue = rescue ? 1u : 0u;
        rec.loc = s.v0;
        rec.ref_lo = s.ref_lo;
        rec.ref_hi = s.ref_hi;
        rec.read_lo = s.read_lo;
        rec.read_hi = s.read_hi;
        o[q] = rec;
      }
    }
    counts[r] = total;
  }
}

// Reads with at most 32 votes: a warp per read, keys sorted in registers.
__global__ void __launch_bounds__(kVT) vote_warp(const god_anchor* __restrict__ a, const uint64_t* __restrict__ read_off,
                                                 const uint64_t* __restrict__ offs, const uint32_t* __restrict__ list,
                                                 const unsigned int* __restrict__ ctl, VoteCfg cfg,
                                                 god_vote_rec* __restrict__ out, uint32_t* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const uint32_t nl = ctl[0];
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t li = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; li < nl; li += warps) {
    const uint32_t r = list[li];
    const uint64_t lo = read_off[r];
    const uint32_t n = (uint32_t)(read_off[r + 1] - lo);
    const uint64_t len = offs[r + 1] - offs[r];
    uint64_t key = ~0ull;
    god_anchor mine{0, 0, 0, 0};
    if ((uint32_t)lane < n) {
      mine = a[lo + lane];
      key = vote_key(mine, len, lane);
    }
    // bitonic sort of 32 keys across the lanes, ascending by lane
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        const uint64_t other = __shfl_xor_sync(kFull, key, j);
        const bool up = (lane & k) == 0;
        const bool lower = (lane & j) == 0;
        const uint64_t lo_v = key < other ? key : other, hi_v = key < other ? other : key;
        key = (lower == up) ? lo_v : hi_v;
      }
    }
    // the anchor behind each sorted key (its index is in the key)
    const uint32_t src = (uint32_t)(key & kIdxMask) & 31u;
    const uint32_t ref = __shfl_sync(kFull, mine.ref_pos, src);
    const uint32_t rp = __shfl_sync(kFull, mine.read_pos, src);
    vote_walk(r, n, cfg,
              [&](uint32_t i, uint64_t* k, uint32_t* rf, uint32_t* p) {
                (void)i;
                *k = key;
                *rf = ref;
                *p = rp;
              },
              out, counts);
  }
}

__device__ void bitonic_smem(uint64_t* s, uint32_t n_pad) {
  for (uint32_t k = 2; k <= n_pad; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint64_t x = s[i], y = s[ixj];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            s[i] = y;
            s[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Loads votes [c0, c1) of a read into s and sorts them (ascending).
__device__ void load_sort_chunk(const god_anchor* __restrict__ a, uint64_t lo, uint64_t len, uint32_t c0, uint32_t c1,
                                uint64_t* s) {
  const uint32_t m = c1 - c0;
  uint32_t n_pad = 1;
  while (n_pad < m) n_pad <<= 1;
  for (uint32_t q = threadIdx.x; q < n_pad; q += blockDim.x)
    s[q] = q < m ? vote_key(a[lo + c0 + q], len, c0 + q) : ~0ull;
  __syncthreads();
  bitonic_smem(s, n_pad);
}

// CTA merge of sorted x[0, nx) and y[0, ny) into o (merge path per thread;
// keys are unique).
__device__ void merge_path(const uint64_t* x, uint64_t nx, const uint64_t* y, uint64_t ny, uint64_t* o) {
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

// Reads with more than 32 votes: a CTA per read, taken from a shared counter
// (lists past 4096 votes first). tmp holds 2 * (votes) keys per chunked read,
// indexed by the read's first anchor.
__global__ void __launch_bounds__(kVT) vote_cta(const god_anchor* __restrict__ a, const uint64_t* __restrict__ read_off,
                                                const uint64_t* __restrict__ offs, const uint32_t* __restrict__ ll,
                                                const uint32_t* __restrict__ lh, unsigned int* ctl, VoteCfg cfg,
                                                uint64_t* tmp, god_vote_rec* __restrict__ out,
                                                uint32_t* __restrict__ counts) {
  __shared__ uint64_t s[kVoteCap];
  __shared__ uint32_t s_li;
  const uint32_t n_long = ctl[1], n_huge = ctl[2];
  const uint32_t nl = n_long + n_huge;
  while (true) {
    if (threadIdx.x == 0) s_li = atomicAdd(ctl + 3, 1u);
    __syncthreads();
    const uint32_t li = s_li;
    __syncthreads();
    if (li >= nl) break;
    const uint32_t r = li < n_huge ? lh[li] : ll[li - n_huge];
    const uint64_t lo = read_off[r];
    const uint32_t n = (uint32_t)(read_off[r + 1] - lo);
    const uint64_t len = offs[r + 1] - offs[r];
    if (n <= kVoteCap) {
      load_sort_chunk(a, lo, len, 0, n, s);
      if (threadIdx.x < 32)
        vote_walk(r, n, cfg,
                  [&](uint32_t i, uint64_t* k, uint32_t* rf, uint32_t* p) {
                    *k = s[i];
                    const god_anchor an = a[lo + (s[i] & kIdxMask)];
                    *rf = an.ref_pos;
                    *p = an.read_pos;
                  },
                  out, counts);
      __syncthreads();
      continue;
    }
    // sorted chunks of kVoteCap in tmp, then merge passes (ping-pong)
    uint64_t* t0 = tmp + 2 * lo;
    uint64_t* t1 = t0 + n;
    for (uint32_t c0 = 0; c0 < n; c0 += kVoteCap) {
      const uint32_t c1 = min(n, c0 + kVoteCap);
      load_sort_chunk(a, lo, len, c0, c1, s);
      for (uint32_t q = threadIdx.x; q < c1 - c0; q += blockDim.x) t0[c0 + q] = s[q];
      __syncthreads();
    }
    uint64_t* x = t0;
    uint64_t* y = t1;
    for (uint64_t run = kVoteCap; run < n; run <<= 1) {
      for (uint64_t j = 0; j < n; j += 2 * run) {
        const uint64_t na = std::min<uint64_t>(run, n - j);
        const uint64_t nb = j + run < n ? std::min<uint64_t>(run, n - j - run) : 0;
        merge_path(x + j, na, x + j + na, nb, y + j);
      }
      __syncthreads();
      uint64_t* t = x;
      x = y;
      y = t;
    }
    if (threadIdx.x < 32)
      vote_walk(r, n, cfg,
                [&](uint32_t i, uint64_t* k, uint32_t* rf, uint32_t* p) {
                  *k = x[i];
                  const god_anchor an = a[lo + (x[i] & kIdxMask)];
                  *rf = an.ref_pos;
                  *p = an.read_pos;
                },
                out, counts);
    __syncthreads();
  }
}

inline unsigned grid_for(uint64_t n, int per, unsigned cap_mult) {
  uint64_t b = (n + per - 1) / per;
  b = std::max<uint64_t>(b, 1);
  return (unsigned)std::min<uint64_t>(b, (uint64_t)num_sms() * cap_mult);
}

}  // namespace

int vote_device(const god_anchor* d_a, uint64_t m, const uint64_t* d_offs, uint32_t n, const god_vote_params& p,
                god_vote_rec* d_out, uint32_t* d_counts, cudaStream_t st) {
  if (n == 0) return GOD_OK;
  const VoteCfg cfg{p.D, p.V, p.max_out};
  DBuf<uint64_t> read_off;
  DBuf<uint32_t> lists;
  DBuf<unsigned int> ctl;
  GOD_TRY(read_off.alloc((uint64_t)n + 1, st));
  GOD_TRY(lists.alloc(4 * (uint64_t)n, st));
  GOD_TRY(ctl.alloc(8, st));
  GOD_CK(cudaMemsetAsync(ctl.p, 0, 8 * sizeof(unsigned int), st));
  int* err = reinterpret_cast<int*>(ctl.p + 4);
  GOD_LAUNCH(vote_ranges, grid_for(m + 1, kVT, 32), kVT, 0, st, d_a, m, n, read_off.p, err);
  uint32_t* lw = lists.p;
  uint32_t* ll = lists.p + n;
  uint32_t* lh = lists.p + 2 * (uint64_t)n;
  uint32_t* lt = lists.p + 3 * (uint64_t)n;
  const uint32_t thread_cap = p.max_out <= kThreadTop ? kVoteThreadCap : 0;
  GOD_LAUNCH(vote_classify, grid_for(n, kVT, 32), kVT, 0, st, n, read_off.p, d_counts, lw, ll, lh, lt, thread_cap,
             ctl.p);
  unsigned int h[8];
  GOD_CK(cudaMemcpyAsync(h, ctl.p, sizeof h, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  if (h[4] == 1) {
    set_error("vote: anchors must be grouped by ascending read id, each below the number of reads");
    return GOD_EINVAL;
  }
  if (h[4] == 2) {
    set_error("vote: a read has 2^28 anchors or more");
    return GOD_EINVAL;
  }
  if (h[5])
    GOD_LAUNCH(vote_thread, grid_for(h[5], kVTT, 24), kVTT, 0, st, d_a, read_off.p, d_offs, lt, ctl.p, cfg, d_out,
               d_counts);
  if (h[0])
    GOD_LAUNCH(vote_warp, grid_for((uint64_t)h[0] * 32, kVT, 16), kVT, 0, st, d_a, read_off.p, d_offs, lw, ctl.p, cfg,
               d_out, d_counts);
  if (h[1] + h[2]) {
    DBuf<uint64_t> tmp;
    if (h[2]) GOD_TRY(tmp.alloc(2 * m, st));
    const unsigned grid = (unsigned)std::min<uint64_t>(h[1] + h[2], (uint64_t)num_sms() * 4);
    GOD_LAUNCH(vote_cta, grid, kVT, 0, st, d_a, read_off.p, d_offs, ll, lh, ctl.p, cfg, tmp.p, d_out, d_counts);
  }
  // algorithmic bytes: one 16-byte anchor read per vote, the read ranges, one
  // record written per reported group
  prof_add_work(h[5] ? "vote_thread" : "vote_warp", 16.0 * (double)m, (double)m);
  return GOD_OK;
}

}  // namespace god
