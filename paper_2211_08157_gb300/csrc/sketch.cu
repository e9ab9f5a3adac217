// Fused seed extraction: sparsify + 2-bit code + canonical Wang hash +
// (w,k)-minimizer selection + ordered compaction, in one persistent kernel.
//
// The method (Sec. 3.1, Sec. 3.6.1) extracts seeds from a patterned sequence:
// keep the bases under the 1s of the repeating diet pattern, code them in 2
// bits (N ends k-mers), hash every canonical k-mer with Thomas Wang's integer
// hash, and keep, in every window of w consecutive k-mers, every k-mer whose
// hash is the window minimum. The paper vectorises this over 8 k-mers with
// AVX-512; here every patterned sequence (the reference, or one read at one
// shift) is a segment of a virtual stream, and CTAs take fixed-size tiles of
// that stream from an atomic ticket, so long and short sequences load-balance
// by construction.
//
// Per tile of T owned k-mer positions [A, A + T):
//  1. gather the 2-bit codes of stream positions [A - w + 1, A + T + w + k - 2)
//     into shared memory; the kept-base arithmetic is closed form
//     (orig = s + p * (j / x) + off[j mod x]), so no scan is needed; a
//     separator position after each segment reads as N;
//  2. roll forward / reverse-complement codes per thread over a contiguous
//     chunk and hash the canonical code -> key + 1 (0 marks a k-mer with N,
//     all-ones marks a palindrome, which is never chosen);
//  3. window minima M[i] = min(key[i .. i + w - 1]) by van Herk / Gil-Werman
//     block prefix/suffix minima;
//  4. position j is a minimizer iff key[j] equals max(M[j - w + 1 .. j]) (every
//     window containing j has minimum <= key[j], so j is some window's minimum
//     exactly when the largest of those minima equals key[j]);
//  5. ordered compaction with a decoupled look-back over tile tickets, so the
//     output is in stream order (segment, position) with no second pass.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace god {
namespace {

constexpr uint64_t kFlagAgg = 1ULL << 62;
constexpr uint64_t kFlagIncl = 2ULL << 62;
constexpr uint64_t kValMask = (1ULL << 62) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;   // ~0.1-1 s of polling before giving up
constexpr uint64_t kPalin = ~0ULL;

__device__ __forceinline__ uint32_t base_code(uint8_t b) {
  const uint32_t c = b & 0xDFu;  // upper-case letters; other bytes stay non-ACGT
  return c == 'A' ? 0u : c == 'C' ? 1u : c == 'G' ? 2u : c == 'T' ? 3u : 4u;
}

// Wang's 64-bit integer hash restricted to 2k bits, written in shift-add form.
// For 2k <= 32 the same steps in 32-bit arithmetic give the identical value.
template <bool WIDE>
__device__ __forceinline__ uint64_t wang_mix(uint64_t key, uint64_t mask) {
  if (WIDE) {
    uint64_t x = key;
    x = (~x + (x << 21)) & mask;
    x = x ^ (x >> 24);
    x = ((x + (x << 3)) + (x << 8)) & mask;
    x = x ^ (x >> 14);
    x = ((x + (x << 2)) + (x << 4)) & mask;
    x = x ^ (x >> 28);
    x = (x + (x << 31)) & mask;
    return x;
  } else {
    uint32_t x = (uint32_t)key;
    const uint32_t m = (uint32_t)mask;
    x = (~x + (x << 21)) & m;
    x = x ^ (x >> 24);
    x = ((x + (x << 3)) + (x << 8)) & m;
    x = x ^ (x >> 14);
    x = ((x + (x << 2)) + (x << 4)) & m;
    x = x ^ (x >> 28);
    x = (x + (x << 31)) & m;
    return x;
  }
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

template <int BLOCK, bool WIDE>
__global__ void __launch_bounds__(BLOCK) sketch_kernel(SketchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const SketchJob& J = a.job;
  const int T = a.T;
  const int k = J.k, w = J.w;
  const int n_keys = T + 2 * (w - 1);
  const int n_codes = n_keys + k - 1;
  const int n_win = T + w - 1;
  // shared layout
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem);
  uint64_t* A1 = keys + n_keys;
  uint64_t* A2 = A1 + n_keys;
  uint32_t* own_seg = reinterpret_cast<uint32_t*>(A2 + n_keys);
  uint32_t* own_pos = own_seg + T;
  uint8_t* codes = reinterpret_cast<uint8_t*>(own_pos + T);
  uint8_t* zb = codes + ((n_codes + 15) & ~15);
  __shared__ uint64_t s_tile_base;
  __shared__ uint32_t s_tile;
  __shared__ uint32_t s_warp_cnt[BLOCK / 32];

  const uint64_t mask = (k >= 32) ? ~0ULL : ((1ULL << (2 * k)) - 1);
  const int rc_shift = 2 * (k - 1);
  const int p = J.pat.p, x = J.pat.x;
  const int tid = threadIdx.x;

  while (true) {
    if (tid == 0) s_tile = atomicAdd(a.ticket, 1u);
    __syncthreads();
    const uint64_t tile = s_tile;
    if (tile >= a.n_tiles) break;
    const int64_t A = (int64_t)(tile * (uint64_t)T);
    const int64_t v_first = A - (w - 1);

    // ---- 1. gather codes (contiguous chunk per thread, incremental segment walk)
    {
      const int R = (n_codes + BLOCK - 1) / BLOCK;
      const int lo = tid * R;
      const int hi = min(lo + R, n_codes);
      bool have = false;
      uint32_t g = 0, j = 0, q = 0, r = 0;
      uint64_t gend = 0;
      SegDesc d{};
      for (int u = lo; u < hi; ++u) {
        const int64_t v = v_first + u;
        uint32_t code = 4;
        const bool own = (u >= w - 1) && (u < w - 1 + T);
        uint32_t oseg = 0xFFFFFFFFu, opos = 0xFFFFFFFFu;
        if (v >= 0 && (uint64_t)v < J.V) {
          if (!have || (uint64_t)v >= gend) {
            g = have ? g + 1 : find_segment(J.seg_voff, J.n_seg, (uint64_t)v);
            d = J.segs[g];
            const uint64_t gstart = J.seg_voff[g];
            gend = J.seg_voff[g + 1];
            j = (uint32_t)((uint64_t)v - gstart);
            q = j / (uint32_t)x;
            r = j - q * (uint32_t)x;
            have = true;
          }
          oseg = g;
          if (j < d.m) {
            const uint64_t orig = (uint64_t)d.shift + (uint64_t)p * q + (uint64_t)J.pat.off[r];
            code = base_code(__ldg(J.bytes + d.byte_off + orig));
            if (code == 4 && (d.flags & kSegCapped) && J.read_flag) J.read_flag[d.read] = 1u;
            opos = (uint32_t)orig;
          }
          ++j;
          if (++r == (uint32_t)x) { r = 0; ++q; }
        }
        codes[u] = (uint8_t)code;
        if (own) {
          own_seg[u - (w - 1)] = oseg;
          own_pos[u - (w - 1)] = opos;
        }
      }
    }
    __syncthreads();

    // ---- 2. canonical k-mer keys (rolling per contiguous chunk)
    {
      const int R = (n_keys + BLOCK - 1) / BLOCK;
      const int lo = tid * R;
      const int hi = min(lo + R, n_keys);
      if (lo < hi) {
        uint64_t fwd = 0, rev = 0;
        int run = 0;
        for (int c = lo; c < lo + k - 1; ++c) {
          const uint32_t b = codes[c];
          if (b == 4) { run = 0; fwd = 0; rev = 0; }
          else {
            ++run;
            fwd = ((fwd << 2) | b) & mask;
            rev = (rev >> 2) | ((uint64_t)(3u - b) << rc_shift);
          }
        }
        for (int i = lo; i < hi; ++i) {
          const uint32_t b = codes[i + k - 1];
          if (b == 4) { run = 0; fwd = 0; rev = 0; }
          else {
            ++run;
            fwd = ((fwd << 2) | b) & mask;
            rev = (rev >> 2) | ((uint64_t)(3u - b) << rc_shift);
          }
          uint64_t kk = 0;
          uint8_t z = 0;
          if (run >= k) {
            if (fwd == rev) kk = kPalin;
            else {
              z = rev < fwd;
              kk = wang_mix<WIDE>(z ? rev : fwd, mask) + 1;
            }
          }
          keys[i] = kk;
          zb[i] = z;
        }
      }
    }
    __syncthreads();

    // ---- 3. window minima (van Herk / Gil-Werman), M -> A1[0 .. n_win)
    {
      const int nb = (n_keys + w - 1) / w;
      for (int b = tid; b < nb; b += BLOCK) {
        const int s = b * w, e = min(s + w, n_keys);
        uint64_t m = ~0ULL;
        for (int i = s; i < e; ++i) { m = min(m, keys[i]); A2[i] = m; }     // prefix
        m = ~0ULL;
        for (int i = e - 1; i >= s; --i) { m = min(m, keys[i]); A1[i] = m; } // suffix
      }
      __syncthreads();
      for (int i = tid; i < n_win; i += BLOCK) A1[i] = min(A1[i], A2[i + w - 1]);
    }
    __syncthreads();

    // ---- 4. largest window minimum containing each owned position
    {
      const int nb = (n_win + w - 1) / w;
      for (int b = tid; b < nb; b += BLOCK) {
        const int s = b * w, e = min(s + w, n_win);
        uint64_t m = 0;
        for (int i = s; i < e; ++i) { m = max(m, A1[i]); A2[i] = m; }      // prefix max
        m = 0;
        for (int i = e - 1; i >= s; --i) { m = max(m, A1[i]); A1[i] = m; } // suffix max (in place)
      }
    }
    __syncthreads();

    // ---- 5. select and compact in stream order
    const int RO = T / BLOCK;  // T is a multiple of BLOCK
    const int o_lo = tid * RO;
    uint32_t sel = 0;  // bit i: owned position o_lo + i is a minimizer (RO <= 32)
    int cnt = 0;
    for (int i = 0; i < RO; ++i) {
      const int o = o_lo + i;
      const uint64_t kk = keys[o + w - 1];
      const uint64_t mx = max(A1[o], A2[o + w - 1]);
      if (kk != 0 && kk != kPalin && kk == mx) { sel |= 1u << i; ++cnt; }
    }
    // block exclusive scan of cnt
    const int lane = tid & 31, wid = tid >> 5;
    int incl = cnt;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, dd);
      if (lane >= dd) incl += y;
    }
    if (lane == 31) s_warp_cnt[wid] = (uint32_t)incl;
    __syncthreads();
    if (tid == 0) {
      uint32_t run = 0;
      for (int i = 0; i < BLOCK / 32; ++i) { const uint32_t c = s_warp_cnt[i]; s_warp_cnt[i] = run; run += c; }
      // decoupled look-back for the tile's global offset
      const uint64_t tile_cnt = run;
      uint64_t excl = 0;
      if (tile == 0) {
        st_release_u64(a.tile_status, kFlagIncl | tile_cnt);
      } else {
        st_release_u64(a.tile_status + tile, kFlagAgg | tile_cnt);
        int64_t pr = (int64_t)tile - 1;
        while (pr >= 0) {
          uint64_t s;
          uint32_t spins = 0;
          while (true) {
            s = ld_acquire_u64(a.tile_status + pr);
            if (s & (kFlagAgg | kFlagIncl)) break;
            if (++spins > kSpinLimit) { atomicExch(a.err, GOD_ETIMEOUT); s = kFlagIncl; break; }
            __nanosleep(64);
          }
          excl += s & kValMask;
          if (s & kFlagIncl) break;
          --pr;
        }
        st_release_u64(a.tile_status + tile, kFlagIncl | (excl + tile_cnt));
      }
      if (tile == a.n_tiles - 1) *a.total = excl + tile_cnt;
      s_tile_base = excl;
    }
    __syncthreads();
    uint64_t dst = s_tile_base + s_warp_cnt[wid] + (uint64_t)(incl - cnt);
    if (sel) {
      for (int i = 0; i < RO; ++i) {
        if (!(sel >> i & 1u)) continue;
        const int o = o_lo + i;
        if (dst < J.out_cap) {
          MinRec rec;
          rec.key = keys[o + w - 1] - 1;
          rec.pos = own_pos[o];
          rec.segz = (own_seg[o] << 1) | zb[o + w - 1];
          J.out[dst] = rec;
        }
        if (J.seg_cnt) atomicAdd(J.seg_cnt + own_seg[o], 1u);
        ++dst;
      }
    }
    __syncthreads();  // shared arrays are rewritten by the next tile
  }
}

size_t sketch_smem_bytes(int T, int k, int w) {
  const size_t n_keys = (size_t)T + 2 * (w - 1);
  const size_t n_codes = n_keys + k - 1;
  return n_keys * 8 * 3 + (size_t)T * 8 + ((n_codes + 15) & ~(size_t)15) + n_keys + 16;
}

template <int BLOCK, bool WIDE>
int launch_sketch_t(const SketchArgs& a, size_t smem, cudaStream_t st) {
  auto sketch = sketch_kernel<BLOCK, WIDE>;
  GOD_CK(cudaFuncSetAttribute(sketch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GOD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sketch, BLOCK, smem));
  if (per_sm < 1) per_sm = 1;
  const uint64_t want = (uint64_t)num_sms() * per_sm;
  const unsigned grid = (unsigned)std::min<uint64_t>(want, a.n_tiles);
  GOD_LAUNCH(sketch, grid, BLOCK, smem, st, a);
  return GOD_OK;
}

}  // namespace

SketchTune default_sketch_tune(int k, int w) {
  (void)k;
  (void)w;
  return SketchTune{2048, 256};
}

int run_sketch(const SketchJob& job, cudaStream_t st, uint64_t* total, const SketchTune* tune) {
  SketchTune tn = tune ? *tune : default_sketch_tune(job.k, job.w);
  if (tn.threads != 128 && tn.threads != 256 && tn.threads != 512) tn.threads = 256;
  if (tn.tile < tn.threads || tn.tile % tn.threads || tn.tile / tn.threads > 32) tn.tile = tn.threads * 8;
  *total = 0;
  if (job.V == 0) return GOD_OK;
  const uint64_t n_tiles = (job.V + tn.tile - 1) / tn.tile;
  // status words + ticket + total + error flag in one allocation
  DBuf<unsigned long long> ws;
  GOD_TRY(ws.alloc(n_tiles + 4, st));
  GOD_CK(cudaMemsetAsync(ws.p, 0, (n_tiles + 4) * sizeof(unsigned long long), st));
  SketchArgs a;
  a.job = job;
  a.tile_status = ws.p;
  a.ticket = reinterpret_cast<unsigned int*>(ws.p + n_tiles);
  a.total = ws.p + n_tiles + 1;
  a.err = reinterpret_cast<int*>(ws.p + n_tiles + 2);
  a.n_tiles = n_tiles;
  a.T = tn.tile;
  const size_t smem = sketch_smem_bytes(tn.tile, job.k, job.w);
  const bool wide = job.k > 16;
  int rc;
  if (tn.threads == 128) rc = wide ? launch_sketch_t<128, true>(a, smem, st) : launch_sketch_t<128, false>(a, smem, st);
  else if (tn.threads == 512) rc = wide ? launch_sketch_t<512, true>(a, smem, st) : launch_sketch_t<512, false>(a, smem, st);
  else rc = wide ? launch_sketch_t<256, true>(a, smem, st) : launch_sketch_t<256, false>(a, smem, st);
  if (rc != GOD_OK) return rc;
  unsigned long long host[3];
  GOD_CK(cudaMemcpyAsync(host, ws.p + n_tiles + 1, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  *total = host[0];
  // algorithmic bytes: every patterned base read once, every record written once
  prof_add_work("sketch", (double)(job.V - job.n_seg) + 16.0 * (double)host[0], (double)(job.V - job.n_seg));
  if ((int)(host[1] & 0xFFFFFFFFu) == GOD_ETIMEOUT) {
    set_error("sketch: ordered-compaction look-back wait gave up");
    return GOD_ETIMEOUT;
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

constexpr uint64_t kNoAllocWords = 32768;                 // 256 KiB of scratch per device
constexpr uint64_t kNoAllocTail = 8;                      // segment descriptor + offsets
constexpr uint64_t kNoAllocMaxTiles = kNoAllocWords - kNoAllocTail - 4;
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
  const SketchTune tn{2048, 256};
  const uint64_t m = patterned_len(P, len, shift);
  const uint64_t V = m + 1;
  const uint64_t n_tiles = (V + tn.tile - 1) / tn.tile;
  if (n_tiles > kNoAllocMaxTiles) {
    set_error("god_sketch_noalloc: patterned length exceeds GOD_NOALLOC_MAX_PATTERNED");
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
  a.ticket = reinterpret_cast<unsigned int*>(scratch + n_tiles);
  a.total = scratch + n_tiles + 1;
  a.err = reinterpret_cast<int*>(scratch + n_tiles + 2);
  a.n_tiles = n_tiles;
  a.T = tn.tile;
  const size_t smem = sketch_smem_bytes(tn.tile, k, w);
  const int lrc = (k > 16) ? launch_sketch_t<256, true>(a, smem, st) : launch_sketch_t<256, false>(a, smem, st);
  if (lrc != GOD_OK) return lrc;
  unsigned long long host[2] = {0, 0};
  GOD_CK(cudaMemcpyAsync(host, scratch + n_tiles + 1, sizeof host, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  *n_out = host[0];
  if ((int)(host[1] & 0xFFFFFFFFu) == GOD_ETIMEOUT) {
    set_error("god_sketch_noalloc: ordered-compaction look-back wait gave up");
    return GOD_ETIMEOUT;
  }
  return host[0] > cap ? GOD_ERANGE : GOD_OK;
}
