// Seed extraction with one thread per short segment (the same minimizers as
// the tile kernel in sketch.cu, for batches whose patterned sequences are all
// short: short reads at every shift, the capped pattern-alignment prefixes of
// long reads).
//
// A warp takes 32 consecutive segments, one per lane. The reference is cut
// into overlapping pieces for this kernel: each piece owns a range of k-mers
// and holds every window that contains one of them, so its minimizers in that
// range are the whole sequence's. When the bytes are in
// page-locked host memory (read over the host link), the warp first loads
// their span (for short reads one contiguous stretch) as aligned 16-byte
// words, coded in 2 bits on the way, into shared memory; device-resident
// bytes, and spans past 4 KB, are read in place through L1 (measured faster
// for device memory: 1.62 against 1.79 ms on 2,000,000 x 150 bp reads). Then each thread walks its segment base by base:
//  * the kept base of patterned index j (orig = s + p (j / x) + off[j mod x],
//    stepped incrementally) is taken in its 2-bit code and rolled into
//    the forward and reverse-complement k-mer codes; a run counter of bases
//    since the last N tells whether the k-mer is usable;
//  * the canonical code is hashed -> key + 1 (0 marks a k-mer with N, all ones
//    a palindrome, which is never chosen), as in the tile kernel;
//  * window minima L[j] = min(key[j - w + 1 .. j]) and the largest covering
//    minimum Y[j] = max(L[j - w + 1 .. j]) come from van Herk / Gil-Werman
//    blocks of w k-mers: the suffix extrema of the previous block are kept in
//    registers (the block loop is unrolled w times, so their indices are
//    constants), the current block's keys and minima in a per-thread
//    shared-memory row, and the running prefix extrema in registers;
//  * k-mer u = j - w + 1 is a minimizer iff it is usable and key[u] = Y[j]
//    (every window holding u has a minimum <= key[u]; u is some window's
//    minimum exactly when the largest of those minima equals key[u]); keys
//    outside the segment are 0, so windows that leave it never decide.
// Records go, in order, to the segment's own slots of the staging array (its
// virtual offset: m + 1 slots >= its k-mers), with the segment's count.
#include <algorithm>

#include "common.cuh"
#include "sketch_common.cuh"

namespace god {
namespace {

constexpr int kSegThreads = 128;
constexpr uint32_t kSegMaxM = 2048;   // longest segment taken by this kernel
constexpr int kWarpBytes = 4096;      // bytes a warp stages for its 32 segments

struct SegArgs {
  SketchJob job;
  MinRec* staging;
  uint32_t* sub_cnt;
};

template <typename KT, int HM, int W, bool STAGE, bool X1, int KC>
__global__ void __launch_bounds__(kSegThreads, (W <= 11 ? 6 : 3)) sketch_seg_kernel(const __grid_constant__ SegArgs a) {
  extern __shared__ __align__(16) unsigned char seg_smem[];
  constexpr int ROW = 2 * W + 1;              // keys B[W], minima C[W]; odd stride: no bank conflicts
  constexpr int WARPS = kSegThreads / 32;
  const unsigned FULL = 0xffffffffu;
  __shared__ uint8_t s_lut[256];
  __shared__ uint32_t s_off[kMaxPattern], s_delta[kMaxPattern];
  const SketchJob& J = a.job;
  // KC > 0: k fixed at compile time (the preset shapes), so the masks, shifts
  // and the palindrome test fold into constants
  const int p = J.pat.p, x = KC && X1 ? 1 : J.pat.x, k = KC ? KC : J.k;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) s_lut[i] = (uint8_t)base_code((uint8_t)i);
  for (int i = threadIdx.x; i < x; i += blockDim.x) {
    s_off[i] = (uint32_t)J.pat.off[i];
    s_delta[i] = (uint32_t)(i + 1 < x ? J.pat.off[i + 1] - J.pat.off[i] : p + J.pat.off[0] - J.pat.off[i]);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  KT* B = reinterpret_cast<KT*>(seg_smem) + threadIdx.x * ROW;
  // the warp's staged bytes, already 2-bit coded (present when staging)
  uint8_t* wcodes = seg_smem + (size_t)kSegThreads * ROW * sizeof(KT) + (size_t)wid * kWarpBytes;
  KT* C = B + W;
  const uint64_t mask = (k >= 32) ? ~0ULL : ((1ULL << (2 * k)) - 1);
  const uint32_t rshift = 2 * k - 2;
  const uint32_t xinv = 0xFFFFFFFFu / (uint32_t)x;
  const KT PALIN = (KT)~(KT)0;
  const uint64_t n_groups = (J.n_seg + 31) / 32;
  const uint64_t warps = (uint64_t)gridDim.x * WARPS;
  // a warp takes 32 consecutive segments, one per lane
  for (uint64_t grp = blockIdx.x * (uint64_t)WARPS + wid; grp < n_groups; grp += warps) {
    const uint64_t g = grp * 32 + lane;
    SegDesc d{0, 0, 0, 0, 0};
    if (g < J.n_seg) d = J.segs[g];
    const uint32_t m = d.m;
    const uint64_t s0 = d.byte_off + d.shift;     // first byte the segment may read
    // one past its last kept base: orig(m - 1) + 1
    uint64_t s1 = s0;
    if (m) {
      uint32_t q, rr;
      divmod_x(m - 1, (uint32_t)x, xinv, q, rr);
      s1 = s0 + (uint64_t)p * q + s_off[rr] + 1;
    }
    // the warp's byte span; staged (coded) in shared memory when it fits
    uint64_t lo = m ? s0 : ~0ull, hi = m ? s1 : 0;
    if (STAGE) {
#pragma unroll
      for (int dd = 16; dd >= 1; dd >>= 1) {
        const uint64_t olo = __shfl_xor_sync(FULL, lo, dd), ohi = __shfl_xor_sync(FULL, hi, dd);
        lo = olo < lo ? olo : lo;
        hi = ohi > hi ? ohi : hi;
      }
    }
    // the span widened to aligned 16-byte words (every such word holds one of
    // the span's bytes, so it lies in a mapped page of the read buffer)
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(J.bytes + lo) & ~(uintptr_t)15;
    const uintptr_t a1 = (reinterpret_cast<uintptr_t>(J.bytes + hi) + 15) & ~(uintptr_t)15;
    const bool staged = STAGE && hi > lo && a1 - a0 <= (uintptr_t)kWarpBytes;
    if (STAGE && staged) {
      const uint32_t nw = (uint32_t)((a1 - a0) >> 4);
      const uint4* wsrc = reinterpret_cast<const uint4*>(a0);
      uint4* wdst = reinterpret_cast<uint4*>(wcodes);
#pragma unroll 4
      for (uint32_t c = lane; c < nw; c += 32) {
        const uint4 v = __ldg(wsrc + c);
        const uint32_t in[4] = {v.x, v.y, v.z, v.w};
        uint32_t outw[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          outw[h] = (uint32_t)s_lut[in[h] & 0xFFu] | ((uint32_t)s_lut[(in[h] >> 8) & 0xFFu] << 8) |
                    ((uint32_t)s_lut[(in[h] >> 16) & 0xFFu] << 16) | ((uint32_t)s_lut[in[h] >> 24] << 24);
        }
        wdst[c] = make_uint4(outw[0], outw[1], outw[2], outw[3]);
      }
    }
    __syncwarp();
    const uint8_t* src = J.bytes + s0;
    const uint8_t* csrc =
        wcodes + (staged && m ? (uint32_t)(reinterpret_cast<uintptr_t>(J.bytes + s0) - a0) : 0u);
    const uint32_t nk = m >= (uint32_t)k ? m - k + 1 : 0;
    uint32_t cnt = 0;
    uint64_t fwd = 0, rev = 0;
    uint32_t run = 0, nflag = 0;
    uint32_t o = s_off[0], r = 0;               // original offset and phase of the next base
    // bases of the first k - 1 positions
    const uint32_t pre = min(m, (uint32_t)k - 1);
    for (uint32_t i = 0; i < pre; ++i) {
      const uint32_t c = (STAGE && staged) ? csrc[o] : s_lut[__ldg(src + o)];
      if (X1) {   // weight-1 pattern: every kept base is p bytes after the last
        o += (uint32_t)p;
      } else {
        o += s_delta[r];
        r = r + 1 == (uint32_t)x ? 0 : r + 1;
      }
      nflag |= c >> 2;
      run = c > 3 ? 0 : run + 1;
      fwd = (fwd << 2) | (c & 3u);
      rev = (rev >> 2) | ((uint64_t)(3u - (c & 3u)) << rshift);
    }
    KT A[W + 1], D[W + 1];                      // suffix minima / maxima of the previous block
#pragma unroll
    for (int t = 0; t <= W; ++t) {
      A[t] = 0;                                 // k-mers before the segment read as 0
      D[t] = 0;
    }
    KT pm = 0, px = 0;
    uint32_t zr = 0;                            // strand bits of the last 32 k-mers (bit 0 = newest)
    MinRec* out = a.staging + (g < J.n_seg ? J.seg_voff[g] : 0);
    uint32_t olo = 0, ohi = 0xFFFFFFFFu;        // owned k-mer indices
    if (J.own && g < J.n_seg) {
      const uint2 ow = reinterpret_cast<const uint2*>(J.own)[g];
      olo = ow.x;
      ohi = ow.y;
    }
    const uint32_t steps = nk ? nk + W - 1 : 0;
    for (uint32_t j0 = 0; j0 < steps; j0 += W) {
#pragma unroll
      for (int t = 0; t < W; ++t) {
        const uint32_t j = j0 + t;
        KT key = 0;
        uint32_t z = 0;
        if (j < nk) {
          const uint32_t c = (STAGE && staged) ? csrc[o] : s_lut[__ldg(src + o)];
          if (X1) {
            o += (uint32_t)p;
          } else {
            o += s_delta[r];
            r = r + 1 == (uint32_t)x ? 0 : r + 1;
          }
          nflag |= c >> 2;
          run = c > 3 ? 0 : run + 1;
          fwd = ((fwd << 2) | (c & 3u)) & mask;
          rev = (rev >> 2) | ((uint64_t)(3u - (c & 3u)) << rshift);
          if (run >= (uint32_t)k) {
            if (!(k & 1) && fwd == rev) {
              key = PALIN;
            } else {
              z = rev < fwd ? 1u : 0u;
              key = (KT)(wang_mix<HM>(z ? rev : fwd, mask) + 1);
            }
          }
        }
        zr = (zr << 1) | z;
        B[t] = key;
        pm = t == 0 ? key : min(pm, key);
        const KT L = t == W - 1 ? pm : min(A[t + 1], pm);
        C[t] = L;
        px = t == 0 ? L : max(px, L);
        const KT Y = t == W - 1 ? px : max(D[t + 1], px);
        if (j >= (uint32_t)W - 1) {
          const KT ku = B[t + 1 < W ? t + 1 : 0];   // key of k-mer u = j - W + 1
          const uint32_t u = j - (W - 1);
          // (odd k: a k-mer is never its own reverse complement)
          if (ku == Y && ku != 0 && ((KC & 1) || ku != PALIN) && u >= olo && u < ohi) {
            uint32_t q = u, rr = 0;
            if (!X1) divmod_x(u, (uint32_t)x, xinv, q, rr);
            MinRec rec;
            rec.key = (uint64_t)ku - 1;
            rec.pos = d.shift + (uint32_t)p * q + s_off[rr];
            rec.segz = ((uint32_t)g << 1) | ((zr >> (W - 1)) & 1u);
            out[cnt++] = rec;
          }
        }
      }
      // this block's suffix extrema for the next block
      A[W - 1] = B[W - 1];
      D[W - 1] = C[W - 1];
#pragma unroll
      for (int t = W - 2; t >= 0; --t) {
        A[t] = min(B[t], A[t + 1]);
        D[t] = max(C[t], D[t + 1]);
      }
    }
    if (g < J.n_seg) {
      a.sub_cnt[g] = cnt;
      if (J.seg_cnt) J.seg_cnt[g] = cnt;
      if (nflag && (d.flags & kSegCapped) && J.read_flag) J.read_flag[d.read] = 1u;
    }
    __syncwarp();   // the staged bytes are rewritten by the next group
  }
}

template <typename KT, int HM, int W, bool STAGE, bool X1, int KC>
int launch_variant(const SegArgs& a, cudaStream_t st) {
  auto sketch_seg = sketch_seg_kernel<KT, HM, W, STAGE, X1, KC>;
  const size_t rows = ((size_t)kSegThreads * (2 * W + 1) * sizeof(KT) + 15) & ~(size_t)15;
  const size_t smem = rows + (STAGE ? (size_t)(kSegThreads / 32) * kWarpBytes : 0);
  GOD_CK(cudaFuncSetAttribute(sketch_seg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GOD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sketch_seg, kSegThreads, smem));
  per_sm = std::max(per_sm, 1);
  const uint64_t need = (a.job.n_seg + kSegThreads - 1) / kSegThreads;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(need, (uint64_t)num_sms() * per_sm));
  GOD_LAUNCH(sketch_seg, grid, kSegThreads, smem, st, a);
  return GOD_OK;
}

// Any k: the pattern weight and the staging choose the variant.
template <typename KT, int HM, int W>
int launch_seg(const SegArgs& a, cudaStream_t st) {
  const bool x1 = a.job.pat.x == 1;
  if (a.job.bytes_on_host)
    return x1 ? launch_variant<KT, HM, W, true, true, 0>(a, st) : launch_variant<KT, HM, W, true, false, 0>(a, st);
  return x1 ? launch_variant<KT, HM, W, false, true, 0>(a, st) : launch_variant<KT, HM, W, false, false, 0>(a, st);
}

// A preset shape with k (and the pattern weight's case) fixed at compile time.
template <typename KT, int HM, int W, int KC, bool X1>
int launch_seg_k(const SegArgs& a, cudaStream_t st) {
  if (a.job.bytes_on_host) return launch_variant<KT, HM, W, true, X1, KC>(a, st);
  return launch_variant<KT, HM, W, false, X1, KC>(a, st);
}

template <int W>
int launch_seg_w(const SegArgs& a, cudaStream_t st) {
  const int k = a.job.k;
  const bool x1 = a.job.pat.x == 1;
  // the preset shapes: k21 w11 and k15 w10 with weight-1 patterns, k19 w19
  // with heavier ones
  if constexpr (W == 11) {
    if (k == 21 && x1) return launch_seg_k<uint64_t, 1, W, 21, true>(a, st);
  } else if constexpr (W == 10) {
    if (k == 15 && x1) return launch_seg_k<uint32_t, 0, W, 15, true>(a, st);
  } else if constexpr (W == 19) {
    if (k == 19 && !x1) return launch_seg_k<uint64_t, 1, W, 19, false>(a, st);
  }
  if (2 * k <= 30) return launch_seg<uint32_t, 0, W>(a, st);
  if (2 * k <= 32) return launch_seg<uint64_t, 0, W>(a, st);
  if (2 * k <= 46) return launch_seg<uint64_t, 1, W>(a, st);
  return launch_seg<uint64_t, 2, W>(a, st);
}

}  // namespace

bool sketch_segments_ok(const SketchJob& job) {
  return job.max_m > 0 && job.max_m <= kSegMaxM && job.n_seg >= 1024 &&
         (job.w == 10 || job.w == 11 || job.w == 19);
}

int run_sketch_segments(const SketchJob& job, cudaStream_t st, StagedSketch& o) {
  o.total = 0;
  o.n_sub = job.n_seg;
  o.WT = 0;
  o.sub_base = job.seg_voff;
  GOD_TRY(o.staging.alloc(job.V, st));
  GOD_TRY(o.sub_cnt.alloc(job.n_seg, st));
  GOD_TRY(o.sub_off.alloc((uint64_t)job.n_seg + 1, st));
  SegArgs a;
  a.job = job;
  a.staging = o.staging.p;
  a.sub_cnt = o.sub_cnt.p;
  if (job.w == 10) GOD_TRY(launch_seg_w<10>(a, st));
  else if (job.w == 11) GOD_TRY(launch_seg_w<11>(a, st));
  else GOD_TRY(launch_seg_w<19>(a, st));
  GOD_TRY(exclusive_scan_u32(o.sub_cnt.p, o.sub_off.p, job.n_seg, st));
  // algorithmic bytes: every patterned base read once, every record written
  // once (the record count is read when the profile is)
  prof_add_work_async("sketch_seg", reinterpret_cast<const unsigned long long*>(o.sub_off.p + job.n_seg),
                      (double)(job.V - job.n_seg), 16.0, (double)(job.V - job.n_seg), 0.0, st);
  return GOD_OK;
}

}  // namespace god
