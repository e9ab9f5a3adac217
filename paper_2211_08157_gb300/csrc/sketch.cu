// Fused seed extraction: sparsify + 2-bit code + canonical Wang hash +
// (w,k)-minimizer selection, in one persistent kernel.
//
// The method (Sec. 3.1, Sec. 3.6.1) extracts seeds from a patterned sequence:
// keep the bases under the 1s of the repeating diet pattern, code them in 2
// bits (N ends k-mers), hash every canonical k-mer with Thomas Wang's integer
// hash, and keep, in every window of w consecutive k-mers, every k-mer whose
// hash is the window minimum. The paper vectorises this over 8 k-mers with
// AVX-512; here every patterned sequence (the reference, or one read at one
// shift) is a segment of a virtual stream, and CTAs stride over fixed-size
// tiles of that stream, so long and short sequences load-balance by
// construction.
//
// Per tile of T owned k-mer positions [A, A + T):
//  1. gather the bases of stream positions [A - w + 1, A + T + w + k - 2)
//     eight per thread through a byte -> 2-bit code table and pack them into
//     64-bit forward and complement words in shared memory; the kept-base
//     arithmetic is closed form (orig = s + p * (j / x) + off[j mod x]), so no
//     scan is needed; a separator position after each segment reads as N;
//  2. four consecutive k-mers per thread from one 64-bit window of each
//     strand; the canonical code is hashed -> key + 1 (0 marks a k-mer with
//     N, all-ones marks a palindrome, which is never chosen);
//  3. window minima M[i] = min(key[i .. i + w - 1]) by van Herk / Gil-Werman
//     block suffix minima (registers) and the next block's prefix minima
//     (shuffles), one warp per sub-tile;
//  4. position j is a minimizer iff key[j] equals max(M[j - w + 1 .. j]) (every
//     window containing j has minimum <= key[j], so j is some window's minimum
//     exactly when the largest of those minima equals key[j]);
//  5. records of the selected positions, in order, into the sub-tile's staging
//     slots (a scan of the per-sub-tile counts orders them), or, for the
//     allocation-free entry point, at their final place after a decoupled
//     look-back over sub-tiles taken from a ticket.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include <cstdio>
#include <cstring>
#include <string>

#include "common.cuh"
#include "sketch_common.cuh"

namespace god {
namespace {

constexpr uint64_t kFlagAgg = 1ULL << 62;
constexpr uint64_t kFlagIncl = 2ULL << 62;
constexpr uint64_t kValMask = (1ULL << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;   // ~0.1-1 s of polling before giving up

// Reverses the order of the 32 two-bit fields of v (field i of the big-endian
// word becomes field i from the bottom, bit order inside a field kept).
__device__ __forceinline__ uint64_t rev_pairs64(uint64_t v) {
  const uint32_t lo = __brev((uint32_t)(v >> 32)), hi = __brev((uint32_t)v);
  const uint32_t lo2 = ((lo >> 1) & 0x55555555u) | ((lo & 0x55555555u) << 1);
  const uint32_t hi2 = ((hi >> 1) & 0x55555555u) | ((hi & 0x55555555u) << 1);
  return ((uint64_t)hi2 << 32) | lo2;
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const unsigned long long* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

struct SketchArgs {
  SketchJob job;
  uint32_t* tile_seg;          // first segment of each CTA tile
  MinRec* staging;             // staged output: WT slots per warp sub-tile
  uint32_t* sub_cnt;           // staged output: records of each sub-tile
  unsigned long long* tile_status;
  unsigned int* ticket;
  unsigned long long* total;
  int* err;
  uint64_t n_tiles;
  int T;
};

__device__ uint32_t find_segment(const uint64_t* voff, uint32_t n_seg, uint64_t v) {
  // largest g with voff[g] <= v
  uint32_t lo = 0, hi = n_seg;  // voff[n_seg] = V > v
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (voff[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// Key storage: 32-bit when 2k <= 30 (key + 1 and the palindrome mark fit),
// 64-bit otherwise. Hash arithmetic: 32-bit when 2k <= 32.
template <typename KT>
__device__ __forceinline__ KT palin_mark() { return (KT)~(KT)0; }

constexpr int kBndCache = 256;  // segment boundaries cached per tile

// Owned positions per warp sub-tile: as many as let `chunks` 8-base chunks per
// thread cover the CTA tile plus its halo (multiple of 8, at least 64).
__host__ __device__ inline int sub_tile_for(int warps, int k, int w, int chunks = 1) {
  int wt = (8 * chunks * 32 * warps - 2 * (w - 1) - (k - 1)) / warps;
  wt &= ~7;
  return wt < 64 ? 64 : wt;
}

// Window stage of the kernel, by variant WV: blocks of exactly WV keys in
// registers (WV > 0: the window lengths of the standard presets, w = 11 and 19
// for 16 < k <= 23 and w = 10 for k <= 15), blocks of up to -WV keys (WV = -12
// or -20), or shared-memory passes for any w (WV = 0).
__host__ __device__ inline int window_variant(int k, int w) {
  if (k > 16 && k <= 23 && (w == 11 || w == 19)) return w;
  if (k <= 15 && w == 10) return w;
  return w <= 12 ? -12 : w <= 20 ? -20 : 0;
}
__host__ __device__ constexpr int window_regs(int wv) { return wv < 0 ? -wv : wv; }

// Shared-memory layout of one CTA tile of T = WARPS * WT owned positions
// (host and device agree on it).
struct TileLayout {
  int n_keys, n_codes, n_groups, n_chunks, n_win_w, warp_scr;
  size_t off_sm, off_f, off_c, off_cst, off_nm, off_vb, off_zb, off_sel, off_list, bytes;
};

__host__ __device__ inline TileLayout tile_layout(int warps, int WT, int k, int w, int kt, int mw) {
  TileLayout L;
  const int T = warps * WT;
  L.n_keys = T + 2 * (w - 1);            // k-mer positions [A - w + 1, A + T + w - 1)
  L.n_codes = L.n_keys + k - 1;          // bases of those k-mers
  L.n_groups = (L.n_codes + 31) / 32;    // 32-base groups (packed words)
  L.n_chunks = L.n_groups * 4;           // 8-base chunks
  L.n_win_w = WT + w - 1;                // windows a warp evaluates
  const int n_keys_w = WT + 2 * (w - 1);
  // per warp: window minima, one column per lane (MW > 0), or S/M and SX
  L.warp_scr = mw > 0 ? mw * 32 : 2 * n_keys_w;
  size_t o = ((size_t)L.n_keys * kt + 15) & ~(size_t)15;        // K (whole tile)
  L.off_sm = o;
  o += (((size_t)L.warp_scr * kt) * warps + 15) & ~(size_t)15;
  L.off_f = o;
  o += (size_t)(L.n_groups + 1) * 8;
  L.off_c = o;
  o += (size_t)(L.n_groups + 1) * 8;
  L.off_cst = o;
  o += (size_t)L.n_chunks * 8;
  L.off_nm = o;
  o += (size_t)(L.n_groups + 1) * 4;
  L.off_vb = o;
  o += (size_t)(L.n_keys / 32 + 3) * 4;  // usable-key bits (key not 0 and not the palindrome mark)
  L.off_zb = o;
  o += (size_t)L.n_keys;
  L.off_sel = o;
  o += mw > 0 ? 0 : (size_t)T;           // selection flags (shared-memory window stage)
  o = (o + 3) & ~(size_t)3;
  L.off_list = o;
  o += (size_t)T * 2;                    // per warp: selected positions (u16)
  L.bytes = (o + 15) & ~(size_t)15;
  return L;
}

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  return v;
}

// 64 bits of a big-endian bit stream {hi64, lo64} starting at bit s (0..63).
__device__ __forceinline__ uint64_t take64_be(uint64_t w0, uint64_t w1, uint32_t s) {
  const uint32_t a = (uint32_t)(w0 >> 32), b = (uint32_t)w0, c = (uint32_t)(w1 >> 32), d = (uint32_t)w1;
  const uint32_t t = s & 31;
  const bool hiw = s >= 32;
  const uint32_t x0 = hiw ? b : a, x1 = hiw ? c : b, x2 = hiw ? d : c;
  const uint32_t hi = __funnelshift_l(x1, x0, t);   // (x0:x1) << t, high word
  const uint32_t lo = __funnelshift_l(x2, x1, t);
  return ((uint64_t)hi << 32) | lo;
}

// 64 bits of a little-endian bit stream {lo64 = w0, hi64 = w1} starting at bit s.
__device__ __forceinline__ uint64_t take64_le(uint64_t w0, uint64_t w1, uint32_t s) {
  const uint32_t a = (uint32_t)w0, b = (uint32_t)(w0 >> 32), c = (uint32_t)w1, d = (uint32_t)(w1 >> 32);
  const uint32_t t = s & 31;
  const bool hiw = s >= 32;
  const uint32_t x0 = hiw ? b : a, x1 = hiw ? c : b, x2 = hiw ? d : c;
  const uint32_t lo = __funnelshift_r(x0, x1, t);   // (x1:x0) >> t, low word
  const uint32_t hi = __funnelshift_r(x1, x2, t);
  return ((uint64_t)hi << 32) | lo;
}

// Window stage with blocks of w <= MW keys in registers (van Herk /
// Gil-Werman): in a pass, lane b takes block b (keys [b w, b w + w) of the
// warp's sub-tile). Its suffix minima stay in registers and the prefix minima
// of block b + 1 come from lane b + 1 by shuffle, giving the window minima that
// start in block b (kept in the lane's own shared-memory column); the same two
// sweeps over those minima give the largest window minimum covering each
// position. Lane b reads keys of blocks b .. b + 2, so a pass completes the
// blocks of lanes 0..29; lanes past the last needed block repeat it. Only the
// windows covering owned positions decide the result, and those lie inside the
// sub-tile's keys, so the reads past its end (still inside the tile's shared
// memory) need no guard. Vb holds the tile's usable-key bits. Appends the
// selected owned positions to `list` in order and returns their number.
template <int MW, typename KT>
__device__ __forceinline__ uint32_t window_select_reg(const KT* __restrict__ Kw, KT* __restrict__ col,
                                                      const uint32_t* __restrict__ Vb, int wo, int w, int WT,
                                                      int lane, uint16_t* __restrict__ list) {
  const unsigned FULL = 0xffffffffu;
  uint32_t cnt = 0;
  const int nb_out = (WT + w - 1) / w;       // blocks holding owned positions
  for (int gb = 0; gb < nb_out; gb += 30) {
    const int s = min(gb + lane, nb_out + 1) * w;
    KT r[MW];
    KT m = palin_mark<KT>();
#pragma unroll
    for (int t = MW - 1; t >= 0; --t) {      // suffix minima of the block
      if (t < w) {
        m = min(m, Kw[s + t]);
        r[t] = m;
      }
    }
    KT pm = palin_mark<KT>();
#pragma unroll
    for (int t = 0; t < MW; ++t) {           // minimum of the window starting at s + t
      if (t < w) {
        KT mv = r[t];
        if (t > 0) mv = min(mv, (KT)__shfl_down_sync(FULL, pm, 1));
        col[t * 32 + lane] = mv;
        pm = min(pm, Kw[s + t]);
      }
    }
    KT mx = 0;
#pragma unroll
    for (int t = MW - 1; t >= 0; --t) {      // suffix maxima of the window minima
      if (t < w) {
        mx = max(mx, col[t * 32 + lane]);
        r[t] = mx;
      }
    }
    KT px = 0;
    uint32_t fl = 0;
#pragma unroll
    for (int t = 0; t < MW; ++t) {           // largest minimum covering s + t, equal to its key?
      if (t < w) {
        KT cover = r[t];
        if (t > 0) cover = max(cover, (KT)__shfl_down_sync(FULL, px, 1));
        if (Kw[s + t + w - 1] == cover) fl |= 1u << t;
        px = max(px, col[t * 32 + lane]);
      }
    }
    // usable keys at s + w - 1 .. s + 2w - 2, owned positions only, lanes 0..29
    const int u0 = wo + s + w - 1;
    fl &= __funnelshift_r(Vb[u0 >> 5], Vb[(u0 >> 5) + 1], u0 & 31);
    const int own = WT - s;
    if (own < 32) fl &= own > 0 ? (1u << own) - 1u : 0u;
    if (lane >= 30 || gb + lane >= nb_out) fl = 0;
    const uint32_t c = __popc(fl);
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, d);
      if (lane >= d) inc += y;
    }
    uint32_t at = cnt + inc - c;
    while (fl) {
      list[at++] = (uint16_t)(s + __ffs(fl) - 1);
      fl &= fl - 1;
    }
    cnt += __shfl_sync(FULL, inc, 31);
  }
  __syncwarp();
  return cnt;
}

// Window stage for any w: the same van Herk / Gil-Werman sweeps with both
// extrema arrays in shared memory (S/M and SX), selection flags, compaction.
template <typename KT>
__device__ __forceinline__ uint32_t window_select_smem(const KT* __restrict__ Kw, KT* SM, KT* SX, uint8_t* sel,
                                                       int w, int n_keys_w, int n_win_w, int WT, int lane,
                                                       uint16_t* __restrict__ list) {
  const KT PALIN = palin_mark<KT>();
  const unsigned FULL = 0xffffffffu;
  {
    const int nb = (n_keys_w + w - 1) / w;
    for (int gb = 0; gb < nb; gb += 31) {
      const int b = gb + lane;
      const int s = b * w;
      const bool live = b < nb;
      KT m = PALIN;
      for (int t = w - 1; t >= 0; --t) {
        const int i = s + t;
        if (live && i < n_keys_w) { m = min(m, Kw[i]); SM[i] = m; }
      }
      __syncwarp();
      KT pm = PALIN;
      for (int t = 0; t < w; ++t) {
        const int i = s + t;
        const KT kv = (live && i < n_keys_w) ? Kw[i] : PALIN;
        const KT nxt = __shfl_down_sync(FULL, pm, 1);   // next block's prefix over offsets < t
        if (lane < 31 && live && i < n_win_w && t) SM[i] = min(SM[i], nxt);
        pm = min(pm, kv);
      }
      __syncwarp();
    }
  }
  {
    const int nb = (n_win_w + w - 1) / w;
    for (int gb = 0; gb < nb; gb += 31) {
      const int b = gb + lane;
      const int s = b * w;
      const bool live = b < nb;
      KT m = 0;
      for (int t = w - 1; t >= 0; --t) {
        const int i = s + t;
        if (live && i < n_win_w) { m = max(m, SM[i]); SX[i] = m; }
      }
      __syncwarp();
      KT px = 0;
      for (int t = 0; t < w; ++t) {
        const int i = s + t;
        const KT mv = (live && i < n_win_w) ? SM[i] : (KT)0;
        const KT nxt = __shfl_down_sync(FULL, px, 1);
        if (lane < 31 && live && i < WT) {
          const KT mx = t == 0 ? SX[i] : max(SX[i], nxt);
          const KT kk = Kw[i + w - 1];
          sel[i] = (kk != 0 && kk != PALIN && kk == mx) ? 1 : 0;
        }
        px = max(px, mv);
      }
      __syncwarp();
    }
  }
  const unsigned lt = (1u << lane) - 1u;
  uint32_t cnt = 0;
  for (int o0 = 0; o0 < WT; o0 += 32) {
    const bool f = o0 + lane < WT && sel[o0 + lane] != 0;
    const unsigned bal = __ballot_sync(FULL, f);
    if (f) list[cnt + __popc(bal & lt)] = (uint16_t)(o0 + lane);
    cnt += __popc(bal);
  }
  __syncwarp();
  return cnt;
}

// Record of the minimizer at tile k-mer index u: its segment from the chunk
// state (walking over segment ends), then the closed-form original position.
template <typename KT>
__device__ __forceinline__ MinRec make_record(const SketchJob& J, const int2* cst, const KT* K, const uint8_t* zb,
                                              int u, uint32_t p, uint32_t x, uint32_t xinv, const uint32_t* s_off,
                                              uint32_t& g_out) {
  const int2 st = cst[u >> 3];
  uint32_t g = (uint32_t)st.x;
  int64_t jj = (int64_t)(uint32_t)st.y - 8 + (u & 7);
  uint32_t m = J.segs[g].m;
  while (jj > (int64_t)m) {
    jj -= (int64_t)m + 1;
    m = J.segs[++g].m;
  }
  uint32_t q, r;
  divmod_x((uint32_t)jj, x, xinv, q, r);
  MinRec rec;
  rec.key = (uint64_t)K[u] - 1;
  rec.pos = J.segs[g].shift + p * q + s_off[r];
  rec.segz = (g << 1) | zb[u];
  g_out = g;
  return rec;
}

// One atomic per distinct segment among the warp's lanes (g = ~0: no record).
__device__ __forceinline__ void count_segments(uint32_t* seg_cnt, uint32_t g, int lane) {
  const unsigned peers = __match_any_sync(0xffffffffu, g);
  if (g != 0xFFFFFFFFu && __ffs(peers) - 1 == lane) atomicAdd(seg_cnt + g, (uint32_t)__popc(peers));
}

// A CTA takes tiles of WARPS * WT positions. All its threads gather, pack and
// hash the tile (one barrier); then each warp evaluates the windows of its own
// WT-position sub-tile and writes its minimizers in order. STAGED: into the
// sub-tile's own WT slots of a staging array plus a count (a scan and a
// compaction pass order them; tiles are strided over CTAs). Otherwise:
// directly to their final place, found by a decoupled look-back over
// sub-tiles taken from a ticket.
template <int WARPS, typename KT, int HM, bool STAGED, int WV>
__global__ void __launch_bounds__(WARPS * 32) sketch_kernel(const __grid_constant__ SketchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int BLOCK = WARPS * 32;
  const int WT = a.T;                         // owned positions per warp
  const int T = WARPS * WT;                   // owned positions per CTA tile
  const SketchJob& J = a.job;
  const int k = J.k, w = J.w;
  constexpr int MW = window_regs(WV);
  const TileLayout Lt = tile_layout(WARPS, WT, k, w, (int)sizeof(KT), MW);
  const int n_keys = Lt.n_keys, n_codes = Lt.n_codes, n_groups = Lt.n_groups, n_chunks = Lt.n_chunks;
  const int n_win_w = Lt.n_win_w;
  const int n_keys_w = WT + 2 * (w - 1);
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  KT* K = reinterpret_cast<KT*>(smem);
  KT* SM = reinterpret_cast<KT*>(smem + Lt.off_sm) + (size_t)wid * Lt.warp_scr;  // this warp's
  uint64_t* F = reinterpret_cast<uint64_t*>(smem + Lt.off_f);
  uint64_t* Cw = reinterpret_cast<uint64_t*>(smem + Lt.off_c);
  int2* cst = reinterpret_cast<int2*>(smem + Lt.off_cst);
  uint32_t* Nm = reinterpret_cast<uint32_t*>(smem + Lt.off_nm);
  uint8_t* zb = smem + Lt.off_zb;
  uint32_t* Vb = reinterpret_cast<uint32_t*>(smem + Lt.off_vb);
  uint16_t* list = reinterpret_cast<uint16_t*>(smem + Lt.off_list) + wid * WT;
  __shared__ uint32_t s_tile, s_gt;
  __shared__ uint32_t bnd[kBndCache + 1];    // seg_voff[g_tile + i] relative to the tile's first base
  __shared__ uint8_t s_lut[256];             // byte -> 2-bit code, 4 for anything but ACGT/acgt
  __shared__ uint32_t s_off[kMaxPattern];    // offsets of the pattern's 1s
  __shared__ uint32_t s_delta[kMaxPattern];  // original-position step to the next kept base

  const uint64_t mask = (k >= 32) ? ~0ULL : ((1ULL << (2 * k)) - 1);
  const uint64_t nmask = (1ULL << k) - 1;
  const uint32_t top_shift = 64 - 2 * k;
  const int p = J.pat.p, x = J.pat.x;
  const uint32_t xinv = 0xFFFFFFFFu / (uint32_t)x;
  const KT PALIN = palin_mark<KT>();
  const unsigned FULL = 0xffffffffu;
  const uint64_t n_sub = a.n_tiles;           // status words are per warp sub-tile
  for (int i = tid; i < 256; i += BLOCK) s_lut[i] = (uint8_t)base_code((uint8_t)i);
  for (int i = tid; i < x; i += BLOCK) {
    s_off[i] = (uint32_t)J.pat.off[i];
    s_delta[i] = (uint32_t)(i + 1 < x ? J.pat.off[i + 1] - J.pat.off[i] : p + J.pat.off[0] - J.pat.off[i]);
  }

  for (uint32_t iter = 0;; ++iter) {
    if (tid == 0) {
      const uint32_t tile = STAGED ? blockIdx.x + iter * gridDim.x : atomicAdd(a.ticket, 1u);
      s_tile = tile;
      s_gt = (uint64_t)tile * WARPS < n_sub ? a.tile_seg[tile] : 0;
    }
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile * WARPS >= n_sub) break;
    const int64_t A = (int64_t)(tile * (uint64_t)T);
    const int64_t v_first = A - (w - 1);
    const uint64_t base_v = v_first < 0 ? 0 : (uint64_t)v_first;
    for (int i = tid; i <= kBndCache; i += BLOCK) {
      const uint64_t bv = J.seg_voff[min((uint64_t)s_gt + i, (uint64_t)J.n_seg)];
      bnd[i] = bv <= base_v ? 0u : (uint32_t)min(bv - base_v, (uint64_t)0xFFFFFFFFu);
    }
    __syncthreads();
    const uint32_t g_tile = s_gt;

    // ---- 1. gather 8 bases per thread step (2-bit codes from the byte table),
    // pack each 32-base group from four lanes
    for (int c0 = 0; c0 < n_chunks; c0 += BLOCK) {
      if (c0 + wid * 32 >= n_chunks) break;   // warp-uniform: whole warp idle
      const int c = c0 + tid;
      const bool act = c < n_chunks;
      const int64_t v0 = v_first + 8 * (int64_t)c;
      uint32_t f16 = 0, n8 = 0xFFu;
      int2 state = make_int2(-1, 0);
      // mode 0: all eight are bases of segment g; 1: rem bases of g, its
      // separator, then bases of g + 1; 2: anything else (stream ends, short
      // segments); 3: no bases
      int mode = 3;
      uint32_t g = 0, j = 0, q = 0, r = 0, rem = 0;
      SegDesc d0{}, d1{};
      if (act && v0 + 8 > 0 && v0 < (int64_t)J.V && 8 * c < n_codes) {
        n8 = 0;
        const uint64_t vs = v0 < 0 ? 0 : (uint64_t)v0;
        const uint32_t vr = (uint32_t)(vs - base_v);
        // segment of vs: the cached boundaries of the tile's first kBndCache
        // segments (global memory only past them)
        if (bnd[kBndCache] <= vr && g_tile + kBndCache < J.n_seg) {
          uint32_t lo = g_tile + kBndCache, hi = J.n_seg;
          while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (J.seg_voff[mid] <= vs) lo = mid; else hi = mid;
          }
          g = lo;
        } else {
          uint32_t lo = 0;
#pragma unroll
          for (int step = kBndCache / 2; step > 0; step >>= 1)
            if (bnd[lo + step] <= vr) lo += step;
          g = g_tile + lo;
        }
        d0 = J.segs[g];
        j = (uint32_t)(vs - J.seg_voff[g]);
        // (segment, index of the chunk's first base in it + 8): biased because
        // the stream's first chunk starts before position 0
        state = make_int2((int)g, (int)(j + 8u - (uint32_t)((int64_t)vs - v0)));
        divmod_x(j, (uint32_t)x, xinv, q, r);
        rem = d0.m - j;
        d1 = d0;
        mode = 2;
        if (v0 >= 0 && 8 * c + 8 <= n_codes) {
          if (rem >= 7) {
            mode = rem >= 8 ? 0 : 1;
          } else if (g + 1 < J.n_seg) {
            d1 = J.segs[g + 1];
            if (6 - rem < d1.m) mode = 1;
          }
        }
      }
      const bool warp_single = __all_sync(FULL, mode == 0 || mode == 3);   // every lane, before branching
      if (mode == 0 && warp_single) {
        // the whole warp inside single segments
        const uint8_t* src = J.bytes + d0.byte_off + d0.shift;
        uint32_t o = (uint32_t)p * q + s_off[r];
        if (x == 1) {
#pragma unroll
          for (int dd = 0; dd < 8; ++dd) {
            const uint32_t e = s_lut[__ldg(src + o + (uint32_t)p * dd)];
            f16 |= (e & 3u) << (14 - 2 * dd);
            n8 |= (e >> 2) << dd;
          }
        } else {
#pragma unroll
          for (int dd = 0; dd < 8; ++dd) {
            const uint32_t e = s_lut[__ldg(src + o)];
            f16 |= (e & 3u) << (14 - 2 * dd);
            n8 |= (e >> 2) << dd;
            o += s_delta[r];
            r = r + 1 == (uint32_t)x ? 0 : r + 1;
          }
        }
        if (n8 && (d0.flags & kSegCapped) && J.read_flag) J.read_flag[d0.read] = 1u;
      } else if (mode <= 1) {
        // segments g and g + 1 walked side by side without branches (mode 0
        // lanes take the same path with every base in g)
        const uint8_t* s0 = J.bytes + d0.byte_off + d0.shift;
        const uint8_t* s1 = J.bytes + d1.byte_off + d1.shift;
        uint32_t o0 = (uint32_t)p * q + s_off[r], r0 = r;
        uint32_t o1 = s_off[0], r1 = 0;
#pragma unroll
        for (int dd = 0; dd < 8; ++dd) {
          const bool in0 = (uint32_t)dd < rem, in1 = (uint32_t)dd > rem;
          const uint32_t b = __ldg((in0 ? s0 + o0 : s1 + o1));   // the separator reads a real base, unused
          const uint32_t e = (in0 || in1) ? s_lut[b] : 4u;
          f16 |= (e & 3u) << (14 - 2 * dd);
          n8 |= (e >> 2) << dd;
          if (x == 1) {
            o0 += in0 ? (uint32_t)p : 0u;
            o1 += in1 ? (uint32_t)p : 0u;
          } else {
            const uint32_t t0 = s_delta[r0], t1 = s_delta[r1];
            if (in0) { o0 += t0; r0 = r0 + 1 == (uint32_t)x ? 0 : r0 + 1; }
            if (in1) { o1 += t1; r1 = r1 + 1 == (uint32_t)x ? 0 : r1 + 1; }
          }
        }
        if (J.read_flag) {   // an N in a capped segment marks its read
          const uint32_t r8 = rem < 8 ? rem : 8u;
          if ((n8 & ((1u << r8) - 1u)) && (d0.flags & kSegCapped)) J.read_flag[d0.read] = 1u;
          if (rem < 7 && (n8 >> (rem + 1)) && (d1.flags & kSegCapped)) J.read_flag[d1.read] = 1u;
        }
      } else if (mode == 2) {
        SegDesc d = d0;
        uint64_t gend = J.seg_voff[g + 1];
        const uint8_t* src = J.bytes + d.byte_off + d.shift;
#pragma unroll
        for (int dd = 0; dd < 8; ++dd) {
          const int64_t v = v0 + dd;
          uint32_t e = 4;
          if (v >= 0 && (uint64_t)v < J.V && 8 * c + dd < n_codes) {
            if ((uint64_t)v >= gend) {
              ++g;
              d = J.segs[g];
              src = J.bytes + d.byte_off + d.shift;
              gend = J.seg_voff[g + 1];
              j = 0; q = 0; r = 0;
            }
            if (j < d.m) {
              e = s_lut[__ldg(src + (uint64_t)p * q + s_off[r])];
              if (e == 4 && (d.flags & kSegCapped) && J.read_flag) J.read_flag[d.read] = 1u;
            }
            ++j;
            if (++r == (uint32_t)x) { r = 0; ++q; }
          }
          f16 |= (e & 3u) << (14 - 2 * dd);
          n8 |= (e >> 2) << dd;
        }
      }
      if (act) cst[c] = state;
      // four consecutive lanes hold the four chunks of one 32-base group
      // (n_chunks is a multiple of 4: a group is all active or all idle)
      const uint32_t v = f16 | (n8 << 16);
      const int gl = lane & ~3;
      const uint32_t v1 = __shfl_sync(FULL, v, gl + 1);
      const uint32_t v2 = __shfl_sync(FULL, v, gl + 2);
      const uint32_t v3 = __shfl_sync(FULL, v, gl + 3);
      if (act && (lane & 3) == 0) {
        const uint64_t fw = ((uint64_t)((v << 16) | (v1 & 0xFFFFu)) << 32) | ((v2 << 16) | (v3 & 0xFFFFu));
        F[c >> 2] = fw;
        Cw[c >> 2] = ~rev_pairs64(fw);   // complements, little-endian (fields under N unused)
        Nm[c >> 2] = (v >> 16) | ((v1 >> 16) << 8) | ((v2 >> 16) << 16) | ((v3 >> 16) << 24);
      }
    }
    if (tid == 0) {  // one spare group so that every k-mer reads two words
      F[n_groups] = 0;
      Cw[n_groups] = 0;
      Nm[n_groups] = 0xFFFFFFFFu;
    }
    if (tid < 3) Vb[n_keys / 32 + tid] = 0;   // words past the last key (rewritten below where keys exist)
    __syncthreads();

    // ---- 2. canonical k-mer keys, four consecutive positions per thread: one
    // 64-bit window of each strand's packed codes (32 bases) holds all four
    const int n_quads = (n_keys + 3) >> 2;
    for (int q0 = 0; q0 < n_quads; q0 += BLOCK) {
      if (q0 + wid * 32 >= n_quads) break;    // warp-uniform
      const int qd = q0 + tid;
      const int i = 4 * qd;
      uint32_t valid4 = 0;
      if (qd < n_quads) {
        const int g = i >> 5, b = i & 31;
        const uint32_t nn = __funnelshift_r(Nm[g], Nm[g + 1], b);
        const uint64_t tb = take64_be(F[g], F[g + 1], 2 * b);   // base i + m at bits 63 - 2m, 62 - 2m
        const uint64_t tl = take64_le(Cw[g], Cw[g + 1], 2 * b);  // its complement at bits 2m, 2m + 1
        KT kq[4];
        uint32_t zq = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          KT kk = 0;
          if (((nn >> j) & (uint32_t)nmask) == 0) {
            uint64_t fwd, rev;
            if (HM > 0) {   // 2k > 32: every shift below is under 32
              const uint32_t sh = top_shift - 2 * j;
              const uint32_t th = (uint32_t)(tb >> 32);
              fwd = ((uint64_t)((th >> sh) & (uint32_t)(mask >> 32)) << 32) | __funnelshift_r((uint32_t)tb, th, sh);
              const uint64_t rs = tl >> (2 * j);
              rev = ((uint64_t)((uint32_t)(rs >> 32) & (uint32_t)(mask >> 32)) << 32) | (uint32_t)rs;
            } else {
              fwd = (uint32_t)(tb >> (top_shift - 2 * j)) & (uint32_t)mask;
              rev = (uint32_t)(tl >> (2 * j)) & (uint32_t)mask;
            }
            if (!(k & 1) && fwd == rev) {   // a palindrome needs even k
              kk = PALIN;
            } else {
              const bool z = rev < fwd;
              zq |= (uint32_t)z << (8 * j);
              kk = (KT)(wang_mix<HM>(z ? rev : fwd, mask) + 1);
              valid4 |= 1u << j;
            }
          }
          kq[j] = kk;
        }
        if (i + 3 < n_keys) {
          if (sizeof(KT) == 8) {
            reinterpret_cast<ulonglong2*>(K + i)[0] = make_ulonglong2(kq[0], kq[1]);
            reinterpret_cast<ulonglong2*>(K + i)[1] = make_ulonglong2(kq[2], kq[3]);
          } else {
            *reinterpret_cast<uint4*>(K + i) = make_uint4((uint32_t)kq[0], (uint32_t)kq[1], (uint32_t)kq[2],
                                                          (uint32_t)kq[3]);
          }
          *reinterpret_cast<uint32_t*>(zb + i) = zq;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (i + j < n_keys) {
              K[i + j] = kq[j];
              zb[i + j] = (uint8_t)(zq >> (8 * j));
            }
          valid4 &= (1u << (n_keys - i)) - 1u;
        }
      }
      // usable-key bits of 32 positions from eight lanes
      uint32_t vb = valid4 << (4 * (lane & 7));
      vb |= __shfl_xor_sync(FULL, vb, 1);
      vb |= __shfl_xor_sync(FULL, vb, 2);
      vb |= __shfl_xor_sync(FULL, vb, 4);
      if ((lane & 7) == 0 && qd < n_quads) Vb[qd >> 3] = vb;
    }
    __syncthreads();

    // ---- 3/4. window minima and the minimizer test over this warp's keys
    // [wo, wo + n_keys_w) of the tile
    const int wo = wid * WT;
    const KT* Kw = K + wo;
    uint32_t cnt;
    if constexpr (MW > 0) {
      cnt = window_select_reg<MW, KT>(Kw, SM, Vb, wo, WV > 0 ? WV : w, WT, lane, list);
    } else {
      cnt = window_select_smem<KT>(Kw, SM, SM + n_keys_w, smem + Lt.off_sel + wid * WT, w, n_keys_w, n_win_w, WT,
                                   lane, list);
    }

    // ---- 5. records of the selected positions, in order: staged per sub-tile,
    // or at their final place after a warp-parallel decoupled look-back
    const uint64_t sub = tile * WARPS + wid;
    uint64_t excl = 0;
    if (STAGED && sub < n_sub) {
      if (lane == 0) a.sub_cnt[sub] = cnt;
      for (uint32_t l0 = 0; l0 < cnt; l0 += 32) {
        const uint32_t li = l0 + lane;
        uint32_t g = 0xFFFFFFFFu;
        if (li < cnt) {
          const MinRec rec = make_record<KT>(J, cst, K, zb, wo + list[li] + w - 1, (uint32_t)p, (uint32_t)x, xinv,
                                             s_off, g);
          a.staging[sub * (uint64_t)WT + li] = rec;
        }
        if (J.seg_cnt) count_segments(J.seg_cnt, g, lane);
      }
    } else if (!STAGED && sub < n_sub) {
      if (sub == 0) {
        if (lane == 0) st_release_u64(a.tile_status, kFlagIncl | cnt);
      } else {
        if (lane == 0) st_release_u64(a.tile_status + sub, kFlagAgg | cnt);
        int64_t pbase = (int64_t)sub - 1;
        while (true) {
          const int64_t idx = pbase - lane;
          uint64_t s = idx >= 0 ? ld_acquire_u64(a.tile_status + idx) : kFlagIncl;
          uint32_t spins = 0;
          while (!__all_sync(FULL, (s & (kFlagAgg | kFlagIncl)) != 0)) {
            if (++spins > kSpinLimit) {
              if (lane == 0) atomicExch(a.err, GOD_ETIMEOUT);
              if (!(s & (kFlagAgg | kFlagIncl))) s = kFlagIncl;
              break;
            }
            __nanosleep(32);
            if (!(s & (kFlagAgg | kFlagIncl))) s = ld_acquire_u64(a.tile_status + idx);
          }
          const unsigned im = __ballot_sync(FULL, (s & kFlagIncl) != 0);
          if (im) {
            const int first = __ffs(im) - 1;          // nearest predecessor with an inclusive prefix
            excl += warp_sum_u64(lane <= first ? (s & kValMask) : 0);
            break;
          }
          excl += warp_sum_u64(s & kValMask);
          pbase -= 32;
        }
        if (lane == 0) st_release_u64(a.tile_status + sub, kFlagIncl | (excl + cnt));
      }
      if (lane == 0 && sub == n_sub - 1) *a.total = excl + cnt;
      for (uint32_t l0 = 0; l0 < cnt; l0 += 32) {
        const uint32_t li = l0 + lane;
        uint32_t g = 0xFFFFFFFFu;
        if (li < cnt) {
          const MinRec rec = make_record<KT>(J, cst, K, zb, wo + list[li] + w - 1, (uint32_t)p, (uint32_t)x, xinv,
                                             s_off, g);
          const uint64_t at = excl + li;
          if (at < J.out_cap) J.out[at] = rec;
        }
        if (J.seg_cnt) count_segments(J.seg_cnt, g, lane);
      }
    }
    __syncthreads();  // the tile's shared memory is rewritten by the next tile
  }
}

template <int WARPS, typename KT, int HM, bool STAGED, int WV>
int launch_sketch_mw(const SketchArgs& a, cudaStream_t st) {
  auto sketch = sketch_kernel<WARPS, KT, HM, STAGED, WV>;
  const size_t smem = tile_layout(WARPS, a.T, a.job.k, a.job.w, (int)sizeof(KT), window_regs(WV)).bytes;
  GOD_CK(cudaFuncSetAttribute(sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GOD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sketch, WARPS * 32, smem));
  if (per_sm < 1) {
    set_error("sketch: tile workspace does not fit in shared memory");
    return GOD_EINVAL;
  }
  const uint64_t want = (uint64_t)num_sms() * per_sm;
  const uint64_t ctas_needed = (a.n_tiles + WARPS - 1) / WARPS;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, ctas_needed));
  GOD_LAUNCH(sketch, grid, WARPS * 32, smem, st, a);
  return GOD_OK;
}

template <int WARPS, typename KT, int HM, bool STAGED>
int launch_sketch_kt(const SketchArgs& a, cudaStream_t st) {
  const int wv = window_variant(a.job.k, a.job.w);
  if constexpr (HM == 1) {
    if (wv == 11) return launch_sketch_mw<WARPS, KT, HM, STAGED, 11>(a, st);
    if (wv == 19) return launch_sketch_mw<WARPS, KT, HM, STAGED, 19>(a, st);
  }
  if constexpr (sizeof(KT) == 4) {
    if (wv == 10) return launch_sketch_mw<WARPS, KT, HM, STAGED, 10>(a, st);
  }
  if (wv == -12) return launch_sketch_mw<WARPS, KT, HM, STAGED, -12>(a, st);
  if (wv == -20) return launch_sketch_mw<WARPS, KT, HM, STAGED, -20>(a, st);
  return launch_sketch_mw<WARPS, KT, HM, STAGED, 0>(a, st);
}

template <int WARPS, bool STAGED>
int launch_sketch_w(const SketchArgs& a, cudaStream_t st) {
  if (a.job.k > 23) return launch_sketch_kt<WARPS, uint64_t, 2, STAGED>(a, st);
  if (a.job.k > 16) return launch_sketch_kt<WARPS, uint64_t, 1, STAGED>(a, st);
  if (a.job.k <= 15) return launch_sketch_kt<WARPS, uint32_t, 0, STAGED>(a, st);
  return launch_sketch_kt<WARPS, uint64_t, 0, STAGED>(a, st);
}

// First segment of every CTA tile (the segment holding its first halo base).
__global__ void tile_first_segment(const uint64_t* voff, uint32_t n_seg, uint64_t V, uint64_t T, int w,
                                   uint64_t n_ctiles, uint32_t* tseg) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n_ctiles; t += (uint64_t)gridDim.x * blockDim.x) {
    const int64_t vf = (int64_t)(t * T) - (w - 1);
    const uint64_t v0 = vf < 0 ? 0 : (uint64_t)vf;
    tseg[t] = v0 < V ? find_segment(voff, n_seg, v0) : 0;
  }
}

// n_tiles in SketchArgs counts warp sub-tiles of a.T positions; the caller
// provides tile_seg for ceil(n_tiles / warps) CTA tiles (or it is computed here).
template <bool STAGED>
int launch_sketch(SketchArgs a, const SketchTune& tn, cudaStream_t st) {
  const int warps = tn.threads / 32;
  const uint64_t n_ctiles = (a.n_tiles + warps - 1) / warps;
  GOD_LAUNCH(tile_first_segment, (unsigned)std::min<uint64_t>((n_ctiles + 255) / 256, 65535), 256, 0, st,
             a.job.seg_voff, a.job.n_seg, a.job.V, (uint64_t)a.T * warps, a.job.w, n_ctiles, a.tile_seg);
  if (tn.threads == 128) {
    if constexpr (STAGED) return launch_sketch_w<4, STAGED>(a, st);
    set_error("sketch: the look-back mode runs 256-thread CTAs");
    return GOD_EINVAL;
  }
  return launch_sketch_w<8, STAGED>(a, st);
}

// Staged records of each sub-tile -> their ordered place (warp per sub-tile).
__global__ void compact_staged(const MinRec* __restrict__ staging, const uint32_t* __restrict__ sub_cnt,
                               const uint64_t* __restrict__ sub_off, uint64_t n_sub, int WT, MinRec* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t sub = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; sub < n_sub; sub += warps) {
    const uint32_t c = sub_cnt[sub];
    const uint64_t o = sub_off[sub];
    const MinRec* src = staging + sub * (uint64_t)WT;
    for (uint32_t i = lane; i < c; i += 32) out[o + i] = src[i];
  }
}

SketchTune clamp_tune(SketchTune tn, int k, int w) {
  if (tn.threads != 128 && tn.threads != 256) tn.threads = 256;
  if (tn.chunks != 1 && tn.chunks != 2) tn.chunks = 1;
  const int kt = k <= 15 ? 4 : 8;
  // shrink until the tile workspace fits one CTA's shared memory
  while (true) {
    tn.tile = sub_tile_for(tn.threads / 32, k, w, tn.chunks);
    if (tile_layout(tn.threads / 32, tn.tile, k, w, kt, window_regs(window_variant(k, w))).bytes + 4096 <= 227 * 1024 ||
        tn.chunks == 1)
      break;
    tn.chunks = 1;
  }
  return tn;
}

// ---- autotuner: launch shape per (k, w, pattern, mean segment length class)
struct TuneEntry {
  SketchTune tn;
  float ms;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, TuneEntry> g_tune;

int len_class(const SketchJob& job) {
  const uint64_t mean = job.n_seg ? job.V / job.n_seg : job.V;
  int c = 0;
  while ((1ull << (c + 1)) <= mean && c < 40) ++c;
  return c;
}

}  // namespace

SketchTune default_sketch_tune(int k, int w) {
  return SketchTune{sub_tile_for(8, k, w), 256, 1};
}

namespace {
struct SketchGraphCtx {
  SketchArgs a;
  SketchTune tn;
  uint64_t* scan_ws;
  uint64_t* sub_off;
  cudaStream_t st;
};
// The persistent sketch pass as one launch sequence: per-tile first segments,
// the sketch kernel, and the scan of the sub-tile counts.
int sketch_pass(void* p) {
  SketchGraphCtx* c = static_cast<SketchGraphCtx*>(p);
  GOD_TRY(launch_sketch<true>(c->a, c->tn, c->st));
  GOD_TRY(exclusive_scan_u32_ws(c->a.sub_cnt, c->sub_off, c->a.n_tiles, c->scan_ws, c->st));
  return GOD_OK;
}

// Staging buffers for one launch shape, allocated before any capture.
struct StageBufs {
  DBuf<uint32_t> tseg;
  DBuf<uint64_t> scan_ws;
};

int prepare(const SketchJob& job, const SketchTune& tn, cudaStream_t st, StagedSketch& o, StageBufs& b,
            SketchGraphCtx& c) {
  const int warps = tn.threads / 32;
  const uint64_t n_sub = (job.V + tn.tile - 1) / tn.tile;
  const uint64_t n_ctiles = (n_sub + warps - 1) / warps;
  o.n_sub = n_sub;
  o.WT = tn.tile;
  GOD_TRY(o.staging.alloc(n_sub * (uint64_t)tn.tile, st));
  GOD_TRY(o.sub_cnt.alloc(n_sub, st));
  GOD_TRY(o.sub_off.alloc(n_sub + 1, st));
  GOD_TRY(b.tseg.alloc(n_ctiles, st));
  GOD_TRY(b.scan_ws.alloc(scan_ws_words(n_sub), st));
  c.a = SketchArgs{};
  c.a.job = job;
  c.a.tile_seg = b.tseg.p;
  c.a.staging = o.staging.p;
  c.a.sub_cnt = o.sub_cnt.p;
  c.a.n_tiles = n_sub;
  c.a.T = tn.tile;
  c.tn = tn;
  c.scan_ws = b.scan_ws.p;
  c.sub_off = o.sub_off.p;
  c.st = st;
  return GOD_OK;
}

// Times each candidate launch shape once on this job (direct launches) and
// returns the fastest; the choice is cached per shape class.
int autotune(const SketchJob& job, cudaStream_t st, SketchTune* best) {
  int dev = 0;
  GOD_CK(cudaGetDevice(&dev));
  const auto key = std::make_tuple(dev, job.k, job.w, job.pat.p * 64 + job.pat.x, len_class(job), (int)(job.seg_cnt != nullptr));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      *best = it->second.tn;
      return GOD_OK;
    }
  }
  const SketchTune cands[4] = {{0, 256, 1}, {0, 128, 1}, {0, 256, 2}, {0, 128, 2}};
  float best_ms = 1e30f;
  SketchTune pick = default_sketch_tune(job.k, job.w);
  cudaEvent_t e0, e1;
  GOD_CK(cudaEventCreate(&e0));
  GOD_CK(cudaEventCreate(&e1));
  for (const SketchTune& cand : cands) {
    const SketchTune tn = clamp_tune(cand, job.k, job.w);
    StagedSketch o;
    StageBufs b;
    SketchGraphCtx c;
    int rc = prepare(job, tn, st, o, b, c);
    if (rc == GOD_OK && job.seg_cnt) rc = cudaMemsetAsync(job.seg_cnt, 0, (size_t)job.n_seg * 4, st) ? GOD_ECUDA : GOD_OK;
    if (rc == GOD_OK) rc = cudaEventRecord(e0, st) ? GOD_ECUDA : GOD_OK;
    if (rc == GOD_OK) rc = sketch_pass(&c);
    if (rc == GOD_OK) rc = cudaEventRecord(e1, st) ? GOD_ECUDA : GOD_OK;
    float ms = 1e30f;
    if (rc == GOD_OK) rc = cudaEventSynchronize(e1) ? GOD_ECUDA : GOD_OK;
    if (rc == GOD_OK) rc = cudaEventElapsedTime(&ms, e0, e1) ? GOD_ECUDA : GOD_OK;
    if (rc != GOD_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc == GOD_ECUDA ? cuda_fail(cudaGetLastError(), "autotune", __FILE__, __LINE__) : rc;
    }
    if (ms < best_ms) {
      best_ms = ms;
      pick = tn;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = TuneEntry{pick, best_ms};
  *best = pick;
  return GOD_OK;
}
}  // namespace

int run_sketch_staged(const SketchJob& job, cudaStream_t st, StagedSketch& o, const SketchTune* tune) {
  SketchTune tn = clamp_tune(tune ? *tune : default_sketch_tune(job.k, job.w), job.k, job.w);
  o.total = 0;
  o.WT = tn.tile;
  o.n_sub = 0;
  if (job.V == 0) {
    GOD_TRY(o.sub_off.alloc(1, st));
    GOD_CK(cudaMemsetAsync(o.sub_off.p, 0, 8, st));
    return GOD_OK;
  }
  if (job.tune && !tune) GOD_TRY(autotune(job, st, &tn));
  StageBufs b;
  SketchGraphCtx c;
  GOD_TRY(prepare(job, tn, st, o, b, c));
  if (job.seg_cnt) GOD_CK(cudaMemsetAsync(job.seg_cnt, 0, (size_t)job.n_seg * 4, st));
  const uint64_t key = ((uint64_t)job.k << 48) ^ ((uint64_t)tn.threads << 36) ^ ((uint64_t)tn.chunks << 32) ^
                       ((uint64_t)(job.seg_cnt != nullptr) << 31) ^ (uint64_t)(job.read_flag != nullptr) ^ 0x5ca1ab1eULL;
  GOD_TRY(graph_run(key, st, sketch_pass, &c));
  uint64_t tot = 0;
  GOD_CK(cudaMemcpyAsync(&tot, o.sub_off.p + o.n_sub, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  GOD_TRY(scan_total_ok(tot, "sketch"));
  o.total = tot;
  // algorithmic bytes: every patterned base read once, every record written once
  prof_add_work("sketch", (double)(job.V - job.n_seg) + 16.0 * (double)tot, (double)(job.V - job.n_seg));
  return GOD_OK;
}

int run_sketch(const SketchJob& job, cudaStream_t st, DBuf<MinRec>& out, uint64_t* total, const SketchTune* tune) {
  StagedSketch S;
  GOD_TRY(run_sketch_staged(job, st, S, tune));
  *total = S.total;
  GOD_TRY(out.alloc(S.total, st));
  if (S.total) {
    const uint64_t blocks = std::min<uint64_t>((S.n_sub * 32 + 255) / 256, (uint64_t)num_sms() * 16);
    GOD_LAUNCH(compact_staged, (unsigned)blocks, 256, 0, st, S.staging.p, S.sub_cnt.p, S.sub_off.p, S.n_sub, S.WT,
               out.p);
  }
  return GOD_OK;
}

}  // namespace god

// ------------------------------------------------------------------------
// Allocation-free sketch entry point (god_sketch_noalloc). Some callers may
// not allocate device memory at all during a call: a host framework whose own
// allocator owns the whole device, a latency-critical loop that cannot take
// the implicit synchronisation of cudaMalloc/cudaFree, or a deployment that
// forbids allocation after start-up. For them the sketch kernel above runs
// with its scratch (look-back status words, tile ticket, total, error flag,
// the one segment descriptor) in a file-scope device array instead of a
// stream-ordered allocation. The array is shared by every call on a device
// and keeps the last call's contents; every word the kernel needs zeroed is
// cleared by a small prep kernel at the start of each call, so calls that
// overlap on the GPU (concurrent streams) race and must be serialised by the
// caller.
namespace god {
namespace {

constexpr uint64_t kNoAllocWords = 262144;                // 2 MiB of scratch per device
constexpr uint64_t kNoAllocTail = 8;                      // segment descriptor + offsets
// Status words (one per sub-tile) + 4 counters + first segment per CTA tile
// (u32, two per word) must fit before the tail. The smallest sub-tile over all
// k <= 28, w <= 255 is sub_tile_for(8, 28, 255) = 184 positions; with it the
// bound below admits patterned lengths up to GOD_NOALLOC_MAX_PATTERNED.
inline bool noalloc_fits(uint64_t n_tiles, uint64_t n_ctiles) {
  return n_tiles + 4 + (n_ctiles + 1) / 2 <= kNoAllocWords - kNoAllocTail;
}
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned long long* g_noalloc_addr[kMaxDevices];          // device address of the array, per device

__global__ void noalloc_prep(unsigned long long* scratch, uint64_t n_tiles, SegDesc seg, uint64_t V) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_tiles + 4;
       i += (uint64_t)gridDim.x * blockDim.x)
    scratch[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *reinterpret_cast<SegDesc*>(scratch + kNoAllocWords - kNoAllocTail) = seg;
    scratch[kNoAllocWords - 2] = 0;   // segment offsets {0, V}
    scratch[kNoAllocWords - 1] = V;
  }
}

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
int noalloc_scratch(unsigned long long** out) {
  int dev = 0;
  GOD_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal out of range");
    return GOD_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
    g_noalloc_addr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_noalloc_addr[dev];
  return GOD_OK;
}

}  // namespace
}  // namespace god

extern "C" int god_sketch_noalloc(const uint8_t* d_seq, uint64_t len, const char* pattern, uint32_t shift, int k,
                                  int w, god_minimizer* d_out, uint64_t cap, uint64_t* n_out, void* stream) {
  using namespace god;
  if (!n_out) return GOD_EINVAL;
  *n_out = 0;
  PatternInfo P;
  if (parse_pattern(pattern, &P) != GOD_OK || k < 1 || k > 28 || w < 1 || w > 255) {
    set_error("god_sketch_noalloc: bad pattern, k or w");
    return GOD_EINVAL;
  }
  if (len >= (1ULL << 32)) {
    set_error("god_sketch_noalloc: sequence must be shorter than 2^32 bases");
    return GOD_EINVAL;
  }
  const SketchTune tn = default_sketch_tune(k, w);
  const uint64_t m = patterned_len(P, len, shift);
  const uint64_t V = m + 1;
  const uint64_t n_tiles = (V + tn.tile - 1) / tn.tile;
  const uint64_t n_ctiles = (n_tiles + tn.threads / 32 - 1) / (tn.threads / 32);
  if (m > GOD_NOALLOC_MAX_PATTERNED || !noalloc_fits(n_tiles, n_ctiles)) {
    set_error("god_sketch_noalloc: patterned length exceeds GOD_NOALLOC_MAX_PATTERNED");
    return GOD_EINVAL;
  }
  // records are written as 16-byte vector stores
  if (cap && (reinterpret_cast<uintptr_t>(d_out) & 15u) != 0) {
    set_error("god_sketch_noalloc: d_out must be 16-byte aligned");
    return GOD_EINVAL;
  }
  if ((len && !is_device_ptr(d_seq)) || (cap && !is_device_ptr(d_out))) {
    set_error("god_sketch_noalloc: sequence and output must be device memory");
    return GOD_EINVAL;
  }
  unsigned long long* scratch = nullptr;
  GOD_TRY(noalloc_scratch(&scratch));
  cudaStream_t st = (cudaStream_t)stream;
  const SegDesc seg{0, (uint32_t)m, 0, shift, 0};
  GOD_LAUNCH(noalloc_prep, (unsigned)std::min<uint64_t>((n_tiles + 4 + 255) / 256, 1024), 256, 0, st, scratch,
             n_tiles, seg, V);
  SketchArgs a;
  a.job = SketchJob{};
  a.job.bytes = d_seq;
  a.job.segs = reinterpret_cast<const SegDesc*>(scratch + kNoAllocWords - kNoAllocTail);
  a.job.seg_voff = reinterpret_cast<const uint64_t*>(scratch + kNoAllocWords - 2);
  a.job.n_seg = 1;
  a.job.V = V;
  a.job.k = k;
  a.job.w = w;
  a.job.pat = P;
  a.job.out = reinterpret_cast<MinRec*>(d_out);   // same 16-byte layout; segment 0 leaves z alone
  a.job.out_cap = cap;
  a.tile_status = scratch;
  a.tile_seg = reinterpret_cast<uint32_t*>(scratch + n_tiles + 4);
  a.ticket = reinterpret_cast<unsigned int*>(scratch + n_tiles);
  a.total = scratch + n_tiles + 1;
  a.err = reinterpret_cast<int*>(scratch + n_tiles + 2);
  a.n_tiles = n_tiles;
  a.T = tn.tile;
  GOD_TRY(launch_sketch<false>(a, tn, st));
  unsigned long long host[2] = {0, 0};
  GOD_CK(cudaMemcpyAsync(host, scratch + n_tiles + 1, sizeof host, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  if ((int)(host[1] & 0xFFFFFFFFu) == GOD_ETIMEOUT) {
    // the total of a pass that gave up means nothing: *n_out stays 0
    set_error("god_sketch_noalloc: ordered-compaction look-back wait gave up");
    return GOD_ETIMEOUT;
  }
  *n_out = host[0];
  return host[0] > cap ? GOD_ERANGE : GOD_OK;
}

extern "C" int god_autotune_report(char* buf, uint64_t cap) {
  using namespace god;
  std::string out = "[";
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    bool first = true;
    for (auto& kv : g_tune) {
      char item[256];
      snprintf(item, sizeof item,
               "%s{\"device\": %d, \"k\": %d, \"w\": %d, \"p\": %d, \"x\": %d, \"len_class\": %d, "
               "\"segment_counts\": %d, \"threads\": %d, \"chunks\": %d, \"tile\": %d, \"ms\": %.4f}",
               first ? "" : ", ", std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
               std::get<3>(kv.first) / 64, std::get<3>(kv.first) % 64, std::get<4>(kv.first), std::get<5>(kv.first),
               kv.second.tn.threads, kv.second.tn.chunks, kv.second.tn.tile, kv.second.ms);
      out += item;
      first = false;
    }
  }
  out += "]";
  if (!buf || cap < out.size() + 1) return (int)(out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return 0;
}
