// Seed matching evaluation (Sec. 2.1.1, Fig. 4): for sequence pairs (S, S'),
// the Levenshtein distance and, for four seeding algorithms, how many seeds
// extracted from S' occur among the seeds extracted from S:
//   0 "All Seeds"       every k-mer (forward 2k-bit code) of A/C/G/T bases;
//   1 "Minimizers"      the (w,k)-minimizer keys of the unsparsified sequence
//                       (canonical k-mers, Wang's hash, all window minima);
//   2 "Spaced"          at every start, the bases under the 1s of the spaced
//                       pattern repeated or cut to k positions (span k);
//   3 "Genome-on-Diet"  every k-mer of the sequence sparsified by the diet
//                       pattern at shift 0.
// Seeds of S' count with repetition. Sequences are at most 1024 bases.
//
// Levenshtein distance: one warp per pair runs Myers' bit-vector recurrence
// (global distance: the top row contributes +1 per column) over a 1024-bit
// column held as one 32-bit word per lane; the carry of the vector addition
// crosses lanes by carry-lookahead on two ballots, the one-bit shifts by a
// shuffle of each lane's top bit.
// Seeds: one CTA per pair builds the four seed arrays of S in shared memory,
// sorts them (bitonic), then every seed of S' is looked up by binary search.
#include <algorithm>

#include "common.cuh"

namespace god {
namespace {

constexpr uint32_t kMaxLen = 1024;
constexpr int kMT = 256;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int code_of(uint8_t c) {
  return c == 'A' || c == 'a' ? 0 : c == 'C' || c == 'c' ? 1 : c == 'G' || c == 'g' ? 2 : c == 'T' || c == 't' ? 3 : 4;
}

// Wang's 64-bit integer hash reduced to 2k bits (a bijection on them).
__device__ __forceinline__ uint64_t wang_hash_bits(uint64_t x, uint64_t mask) {
  x = (x * 0x1FFFFFull + ~0ull) & mask;
  x ^= x >> 24;
  x = (x * 265ull) & mask;
  x ^= x >> 14;
  x = (x * 21ull) & mask;
  x ^= x >> 28;
  x = (x * 0x80000001ull) & mask;
  return x;
}

__global__ void __launch_bounds__(kMT) levenshtein_warp(const uint8_t* __restrict__ seqs,
                                                        const uint64_t* __restrict__ offs, uint32_t n,
                                                        uint32_t* __restrict__ ed, int* err) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t i = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; i < n; i += warps) {
    const uint64_t a0 = offs[2 * i], a1 = offs[2 * i + 1], b1 = offs[2 * i + 2];
    if (a1 < a0 || b1 < a1 || a1 - a0 > kMaxLen || b1 - a1 > kMaxLen) {
      if (lane == 0) atomicExch(err, 1);
      continue;
    }
    const uint32_t m = (uint32_t)(a1 - a0), nt = (uint32_t)(b1 - a1);
    const uint8_t* S = seqs + a0;
    const uint8_t* T = seqs + a1;
    if (m == 0) {
      if (lane == 0) ed[i] = nt;
      continue;
    }
    // match masks of this lane's 32 pattern positions for A, C, G, T
    uint32_t peq[4] = {0, 0, 0, 0};
    for (int b = 0; b < 32; ++b) {
      const uint32_t q = (uint32_t)lane * 32 + b;
      if (q < m) {
        const uint8_t c = S[q];
        if (c == 'A') peq[0] |= 1u << b;
        else if (c == 'C') peq[1] |= 1u << b;
        else if (c == 'G') peq[2] |= 1u << b;
        else if (c == 'T') peq[3] |= 1u << b;
      }
    }
    const int last_lane = (int)((m - 1) >> 5);
    const uint32_t last_bit = 1u << ((m - 1) & 31);
    uint32_t Pv = kFull, Mv = 0;
    int score = (int)m;
    for (uint32_t j = 0; j < nt; ++j) {
      const uint8_t t = T[j];
      uint32_t Eq;
      if (t == 'A') Eq = peq[0];
      else if (t == 'C') Eq = peq[1];
      else if (t == 'G') Eq = peq[2];
      else if (t == 'T') Eq = peq[3];
      else {
        Eq = 0;
        for (int b = 0; b < 32; ++b) {
          const uint32_t q = (uint32_t)lane * 32 + b;
          if (q < m && S[q] == t) Eq |= 1u << b;
        }
      }
      const uint32_t Xv = Eq | Mv;
      // (Eq & Pv) + Pv over the whole column: per-lane sums, then the carries
      // into each lane from generate / propagate ballots
      const uint32_t x = Eq & Pv;
      uint32_t s = x + Pv;
      const unsigned G = __ballot_sync(kFull, s < x);
      const unsigned Pr = __ballot_sync(kFull, s == kFull);
      const unsigned GP = G | Pr;
      const unsigned C = (G + GP) ^ G ^ GP;
      s += (C >> lane) & 1u;
      const uint32_t Xh = (s ^ Pv) | Eq;
      uint32_t Ph = Mv | ~(Xh | Pv);
      uint32_t Mh = Pv & Xh;
      if (lane == last_lane) score += (Ph & last_bit) ? 1 : ((Mh & last_bit) ? -1 : 0);
      uint32_t ph_in = __shfl_up_sync(kFull, Ph >> 31, 1);
      uint32_t mh_in = __shfl_up_sync(kFull, Mh >> 31, 1);
      if (lane == 0) {
        ph_in = 1u;   // row 0 of the table grows by one per column
        mh_in = 0u;
      }
      Ph = (Ph << 1) | ph_in;
      Mh = (Mh << 1) | mh_in;
      Pv = Mh | ~(Xv | Ph);
      Mv = Ph & Xv;
    }
    score = __shfl_sync(kFull, score, last_lane);
    if (lane == 0) ed[i] = (uint32_t)score;
  }
}

struct MatchCfg {
  int k, w;
  int sp_n;                  // spaced seed: number of read offsets
  int sp_off[28];            // offsets (< k) of the spaced pattern's 1s
  PatternInfo P;             // diet pattern
};

// Code of the bases at s[pos + off[t]] (t < q); ~0 if one is not A/C/G/T.
__device__ __forceinline__ uint64_t gapped_code(const uint8_t* s, uint32_t pos, const int* off, int q) {
  uint64_t v = 0;
  for (int t = 0; t < q; ++t) {
    const int c = code_of(s[pos + off[t]]);
    if (c == 4) return ~0ull;
    v = (v << 2) | (uint64_t)c;
  }
  return v;
}

// Original index of patterned base j (shift 0).
__device__ __forceinline__ uint32_t kept_pos(const PatternInfo& P, uint32_t j) {
  return (uint32_t)P.p * (j / (uint32_t)P.x) + (uint32_t)P.off[j % (uint32_t)P.x];
}

__device__ __forceinline__ uint64_t god_code(const uint8_t* s, const PatternInfo& P, uint32_t j, int k) {
  uint64_t v = 0;
  for (int t = 0; t < k; ++t) {
    const int c = code_of(s[kept_pos(P, j + t)]);
    if (c == 4) return ~0ull;
    v = (v << 2) | (uint64_t)c;
  }
  return v;
}

// Minimizer flags of s (length L): key[i] and chosen[i] for k-mer start i.
__device__ void minimizer_flags(const uint8_t* s, uint32_t L, int k, int w, uint64_t* key, uint8_t* state,
                                uint8_t* chosen) {
  const uint32_t nk = L >= (uint32_t)k ? L - k + 1 : 0;
  const uint64_t mask = k == 32 ? ~0ull : ((1ull << (2 * k)) - 1);
  // state: 0 = N inside, 1 = usable, 2 = usable palindrome
  for (uint32_t i = threadIdx.x; i < nk; i += blockDim.x) {
    uint64_t f = 0, r = 0;
    bool ok = true;
    for (int t = 0; t < k; ++t) {
      const int c = code_of(s[i + t]);
      if (c == 4) { ok = false; break; }
      f = (f << 2) | (uint64_t)c;
      r |= (uint64_t)(3 - c) << (2 * t);
    }
    chosen[i] = 0;
    if (!ok) { state[i] = 0; continue; }
    state[i] = f == r ? 2 : 1;
    key[i] = wang_hash_bits(f < r ? f : r, mask);
  }
  __syncthreads();
  for (uint32_t st = threadIdx.x; st + w <= nk; st += blockDim.x) {
    bool ok = true, have = false;
    uint64_t mn = 0;
    for (uint32_t j = st; j < st + (uint32_t)w; ++j) {
      if (state[j] == 0) { ok = false; break; }
      if (state[j] == 1 && (!have || key[j] < mn)) { mn = key[j]; have = true; }
    }
    if (!ok || !have) continue;
    for (uint32_t j = st; j < st + (uint32_t)w; ++j)
      if (state[j] == 1 && key[j] == mn) chosen[j] = 1;
  }
  __syncthreads();
}

__device__ void bitonic1024(uint64_t* a) {
  for (uint32_t kk = 2; kk <= kMaxLen; kk <<= 1) {
    for (uint32_t j = kk >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < kMaxLen; i += blockDim.x) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint64_t x = a[i], y = a[ixj];
          const bool up = (i & kk) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

__device__ __forceinline__ bool in_sorted(const uint64_t* a, uint64_t v) {
  uint32_t lo = 0, hi = kMaxLen;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo < kMaxLen && a[lo] == v;
}

__global__ void __launch_bounds__(kMT) seed_match_cta(const uint8_t* __restrict__ seqs,
                                                      const uint64_t* __restrict__ offs, uint32_t n, MatchCfg cfg,
                                                      uint32_t* __restrict__ matched, uint32_t* __restrict__ total) {
  __shared__ uint64_t sorted[4][kMaxLen];
  __shared__ uint64_t key[kMaxLen];
  __shared__ uint8_t state[kMaxLen], chosen[kMaxLen];
  __shared__ uint8_t sa[kMaxLen], sb[kMaxLen];
  __shared__ uint32_t cnt[8];
  const int k = cfg.k;
  int contig[28];
  for (int t = 0; t < 28; ++t) contig[t] = t;
  for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
    const uint64_t a0 = offs[2 * i], a1 = offs[2 * i + 1], b1 = offs[2 * i + 2];
    if (a1 < a0 || b1 < a1 || a1 - a0 > kMaxLen || b1 - a1 > kMaxLen) continue;   // flagged by the distance kernel
    const uint32_t la = (uint32_t)(a1 - a0), lb = (uint32_t)(b1 - a1);
    for (uint32_t q = threadIdx.x; q < la; q += blockDim.x) sa[q] = seqs[a0 + q];
    for (uint32_t q = threadIdx.x; q < lb; q += blockDim.x) sb[q] = seqs[a1 + q];
    if (threadIdx.x < 8) cnt[threadIdx.x] = 0;
    for (uint32_t q = threadIdx.x; q < 4 * kMaxLen; q += blockDim.x) sorted[q / kMaxLen][q % kMaxLen] = ~0ull;
    __syncthreads();
    // seeds of S
    const uint32_t na = la >= (uint32_t)k ? la - k + 1 : 0;
    const uint32_t ma = (uint32_t)patterned_len(cfg.P, la, 0);
    const uint32_t ga = ma >= (uint32_t)k ? ma - k + 1 : 0;
    for (uint32_t q = threadIdx.x; q < na; q += blockDim.x) {
      sorted[0][q] = gapped_code(sa, q, contig, k);
      sorted[2][q] = gapped_code(sa, q, cfg.sp_off, cfg.sp_n);
    }
    for (uint32_t q = threadIdx.x; q < ga; q += blockDim.x) sorted[3][q] = god_code(sa, cfg.P, q, k);
    minimizer_flags(sa, la, k, cfg.w, key, state, chosen);
    for (uint32_t q = threadIdx.x; q < na; q += blockDim.x)
      if (chosen[q]) sorted[1][q] = key[q];
    __syncthreads();
    for (int g = 0; g < 4; ++g) bitonic1024(sorted[g]);
    // seeds of S', looked up
    const uint32_t nb = lb >= (uint32_t)k ? lb - k + 1 : 0;
    const uint32_t mb = (uint32_t)patterned_len(cfg.P, lb, 0);
    const uint32_t gb = mb >= (uint32_t)k ? mb - k + 1 : 0;
    uint32_t hit[4] = {0, 0, 0, 0}, tot[4] = {0, 0, 0, 0};
    for (uint32_t q = threadIdx.x; q < nb; q += blockDim.x) {
      uint64_t v = gapped_code(sb, q, contig, k);
      if (v != ~0ull) { ++tot[0]; hit[0] += in_sorted(sorted[0], v); }
      v = gapped_code(sb, q, cfg.sp_off, cfg.sp_n);
      if (v != ~0ull) { ++tot[2]; hit[2] += in_sorted(sorted[2], v); }
    }
    for (uint32_t q = threadIdx.x; q < gb; q += blockDim.x) {
      const uint64_t v = god_code(sb, cfg.P, q, k);
      if (v != ~0ull) { ++tot[3]; hit[3] += in_sorted(sorted[3], v); }
    }
    minimizer_flags(sb, lb, k, cfg.w, key, state, chosen);
    for (uint32_t q = threadIdx.x; q < nb; q += blockDim.x)
      if (chosen[q]) { ++tot[1]; hit[1] += in_sorted(sorted[1], key[q]); }
    for (int g = 0; g < 4; ++g) {
      uint32_t h = hit[g], t = tot[g];
      for (int d = 16; d >= 1; d >>= 1) {
        h += __shfl_xor_sync(kFull, h, d);
        t += __shfl_xor_sync(kFull, t, d);
      }
      if ((threadIdx.x & 31) == 0) {
        atomicAdd(&cnt[g], h);
        atomicAdd(&cnt[4 + g], t);
      }
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      matched[4 * (uint64_t)i + threadIdx.x] = cnt[threadIdx.x];
      total[4 * (uint64_t)i + threadIdx.x] = cnt[4 + threadIdx.x];
    }
    __syncthreads();
  }
}

inline unsigned grid_for(uint64_t n, int per, unsigned cap_mult) {
  uint64_t b = (n + per - 1) / per;
  b = std::max<uint64_t>(b, 1);
  return (unsigned)std::min<uint64_t>(b, (uint64_t)num_sms() * cap_mult);
}

}  // namespace

int seed_match_device(const uint8_t* d_seqs, const uint64_t* d_offs, uint32_t n, const PatternInfo& P,
                      const PatternInfo& SP, int k, int w, uint32_t* d_ed, uint32_t* d_matched, uint32_t* d_total,
                      cudaStream_t st) {
  if (n == 0) return GOD_OK;
  MatchCfg cfg{};
  cfg.k = k;
  cfg.w = w;
  cfg.P = P;
  cfg.sp_n = 0;
  for (int i = 0; i < k; ++i) {
    const int ph = i % SP.p;
    if (SP.ones_prefix[ph + 1] != SP.ones_prefix[ph]) cfg.sp_off[cfg.sp_n++] = i;
  }
  DBuf<int> err;
  GOD_TRY(err.alloc(1, st));
  GOD_CK(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  GOD_LAUNCH(levenshtein_warp, grid_for((uint64_t)n * 32, kMT, 16), kMT, 0, st, d_seqs, d_offs, n, d_ed, err.p);
  GOD_LAUNCH(seed_match_cta, (unsigned)std::min<uint64_t>(n, (uint64_t)num_sms() * 4), kMT, 0, st, d_seqs, d_offs, n,
             cfg, d_matched, d_total);
  int herr = 0;
  GOD_CK(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  if (herr) {
    set_error("seed match: each sequence must be at most 1024 bases, offsets non-decreasing");
    return GOD_EINVAL;
  }
  return GOD_OK;
}

}  // namespace god
