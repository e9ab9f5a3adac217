// Segmented seeding: reads longer than a segment length S are cut into
// consecutive segments [j S, (j + 1) S) (the last one shorter), the way the
// paper splits ultra-long reads into segments of at most 30,000 bases
// (Sec. 2.2.2). Every segment is pattern-aligned on its own (Sec. 3.2: its own
// shift, so the phase lost after an indel is found again in the next segment)
// and seeded like a read by the batched pipeline; its anchors then carry the
// read's id and whole-read positions, and a read's per-segment sorted runs
// are merged into one list sorted by (ref_pos, read_pos, strand).
#include <algorithm>

#include "common.cuh"

namespace god {
namespace {

constexpr int kST = 256;

inline unsigned grid_for(uint64_t n, int per, unsigned cap_mult) {
  uint64_t b = (n + per - 1) / per;
  b = std::max<uint64_t>(b, 1);
  return (unsigned)std::min<uint64_t>(b, (uint64_t)num_sms() * cap_mult);
}

__device__ __forceinline__ uint32_t seg_count_of(uint64_t len, uint32_t S) {
  return len <= S ? 1u : (uint32_t)((len + S - 1) / S);
}

// Segments per read (err = 1 on decreasing offsets or a read of 2^31 bytes or more).
__global__ void seg_count(const uint64_t* __restrict__ offs, uint32_t n, uint32_t S, uint32_t* __restrict__ nseg,
                          int* err) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = offs[r], e = offs[r + 1];
    uint64_t len = e - b;
    if (e < b || len >= (1ull << 31)) {
      atomicExch(err, 1);
      len = 0;
    }
    nseg[r] = seg_count_of(len, S);
  }
}

// CSR byte offsets of the segments, their owning read and start inside it.
__global__ void seg_fill(const uint64_t* __restrict__ offs, uint32_t n, uint32_t S, const uint64_t* __restrict__ first,
                         uint64_t* __restrict__ soff, uint32_t* __restrict__ sown) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = offs[r];
    const uint64_t f = first[r], c = first[r + 1] - f;
    for (uint64_t j = 0; j < c; ++j) {
      soff[f + j] = b + j * S;
      sown[f + j] = (uint32_t)r;
    }
    if (r == n - 1) soff[f + c] = offs[n];
  }
}

// Anchor ranges per segment: seg_aoff[s] = first anchor whose (segment) id is >= s.
__global__ void seg_anchor_ranges(const god_anchor* __restrict__ a, uint64_t m, uint64_t N,
                                  uint64_t* __restrict__ seg_aoff) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t cur = i < m ? (uint64_t)a[i].read_id : N;
    const uint64_t lo = i > 0 ? (uint64_t)a[i - 1].read_id + 1 : 0;
    for (uint64_t s = lo; s <= cur && s <= N; ++s) seg_aoff[s] = i;
  }
}

// Segment ids -> read ids, segment positions -> read positions.
__global__ void seg_remap(god_anchor* __restrict__ a, uint64_t m, const uint64_t* __restrict__ soff,
                          const uint32_t* __restrict__ sown, const uint64_t* __restrict__ offs) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = a[i].read_id;
    const uint32_t r = sown[s];
    a[i].read_id = r;
    a[i].read_pos += (uint32_t)(soff[s] - offs[r]);
  }
}

__global__ void seg_list_split(uint32_t n, const uint64_t* __restrict__ first, uint32_t* __restrict__ list,
                               unsigned int* counter) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    if (first[r + 1] - first[r] > 1) list[atomicAdd(counter, 1u)] = (uint32_t)r;
  }
}

__device__ __forceinline__ uint64_t akey(const god_anchor& x) {
  return ((uint64_t)x.ref_pos << 32) | ((uint64_t)x.read_pos << 1) | (x.strand & 1u);
}

// CTA merge of sorted x[0, nx) and y[0, ny) into o (keys unique inside a read).
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

// A CTA per split read: its segments' sorted runs are merged one after the
// other (run 0 with run 1, the result with run 2, ...) in tmp, indexed by the
// read's first anchor (2 keys per anchor), then written back.
__global__ void __launch_bounds__(kST) seg_merge(god_anchor* __restrict__ a, const uint64_t* __restrict__ seg_aoff,
                                                 const uint64_t* __restrict__ first,
                                                 const uint32_t* __restrict__ list, const unsigned int* counter,
                                                 uint64_t* tmp) {
  const uint32_t nl = *counter;
  for (uint32_t li = blockIdx.x; li < nl; li += gridDim.x) {
    const uint32_t r = list[li];
    const uint64_t s0 = first[r], s1 = first[r + 1];
    const uint64_t lo = seg_aoff[s0], hi = seg_aoff[s1];
    const uint64_t n = hi - lo;
    if (n == 0) continue;
    uint64_t* x = tmp + 2 * lo;
    uint64_t* y = x + n;
    for (uint64_t q = threadIdx.x; q < n; q += blockDim.x) x[q] = akey(a[lo + q]);
    __syncthreads();
    uint64_t acc = seg_aoff[s0 + 1] - lo;   // merged prefix length
    for (uint64_t s = s0 + 1; s < s1; ++s) {
      const uint64_t run = seg_aoff[s + 1] - seg_aoff[s];
      if (run) {
        merge_path(x, acc, x + acc, run, y);
        __syncthreads();
        for (uint64_t q = threadIdx.x; q < acc + run; q += blockDim.x) x[q] = y[q];
        __syncthreads();
      }
      acc += run;
    }
    for (uint64_t q = threadIdx.x; q < n; q += blockDim.x) {
      const uint64_t k = x[q];
      god_anchor o;
      o.read_id = r;
      o.read_pos = (uint32_t)(k >> 1) & 0x7FFFFFFFu;
      o.ref_pos = (uint32_t)(k >> 32);
      o.strand = (uint32_t)(k & 1u);
      a[lo + q] = o;
    }
    __syncthreads();
  }
}

}  // namespace

int seed_segmented(const god_index* idx, const uint8_t* d_reads, const uint64_t* d_offs, uint32_t n,
                   uint64_t read_bytes, const god_seed_opts& o, cudaStream_t st, god_anchor** d_out,
                   uint64_t* n_anchors, god_anchor* user_out, uint64_t user_cap, bool user_out_device) {
  const uint32_t S = o.seg_len;
  god_seed_opts o2 = o;
  o2.seg_len = 0;
  *n_anchors = 0;
  if (n == 0) return GOD_OK;
  DBuf<uint32_t> nseg;
  DBuf<uint64_t> first;
  DBuf<int> err;
  GOD_TRY(nseg.alloc(n, st));
  GOD_TRY(first.alloc((uint64_t)n + 1, st));
  GOD_TRY(err.alloc(1, st));
  GOD_CK(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  GOD_LAUNCH(seg_count, grid_for(n, kST, 32), kST, 0, st, d_offs, n, S, nseg.p, err.p);
  GOD_TRY(exclusive_scan_u32(nseg.p, first.p, n, st));
  uint64_t N = 0;
  int herr = 0;
  GOD_CK(cudaMemcpyAsync(&N, first.p + n, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  if (herr) {
    set_error("seed: offsets must be non-decreasing and each read < 2^31 bytes");
    return GOD_EINVAL;
  }
  GOD_TRY(scan_total_ok(N, "seed"));
  if (N == n)   // no read is longer than a segment
    return seed_device(idx, d_reads, d_offs, n, read_bytes, o2, st, d_out, n_anchors, user_out, user_cap,
                       user_out_device);
  if (N >= (1ull << 31)) {
    set_error("seed: too many segments");
    return GOD_EINVAL;
  }
  DBuf<uint64_t> soff;
  DBuf<uint32_t> sown;
  GOD_TRY(soff.alloc(N + 1, st));
  GOD_TRY(sown.alloc(N, st));
  GOD_LAUNCH(seg_fill, grid_for(n, kST, 32), kST, 0, st, d_offs, n, S, first.p, soff.p, sown.p);
  uint64_t m = 0;
  const int rc = seed_device(idx, d_reads, soff.p, (uint32_t)N, read_bytes, o2, st, d_out, &m, user_out, user_cap,
                             user_out_device);
  *n_anchors = m;   // also the needed count on GOD_ERANGE
  if (rc != GOD_OK) return rc;
  if (m == 0) return GOD_OK;
  god_anchor* a = user_out ? user_out : *d_out;
  DBuf<uint64_t> seg_aoff;
  DBuf<uint32_t> list;
  DBuf<unsigned int> cnt;
  DBuf<uint64_t> tmp;
  GOD_TRY(seg_aoff.alloc(N + 1, st));
  GOD_TRY(list.alloc(n, st));
  GOD_TRY(cnt.alloc(1, st));
  GOD_TRY(tmp.alloc(2 * m, st));
  GOD_CK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned int), st));
  GOD_LAUNCH(seg_anchor_ranges, grid_for(m + 1, kST, 32), kST, 0, st, a, m, N, seg_aoff.p);
  GOD_LAUNCH(seg_remap, grid_for(m, kST, 32), kST, 0, st, a, m, soff.p, sown.p, d_offs);
  GOD_LAUNCH(seg_list_split, grid_for(n, kST, 32), kST, 0, st, n, first.p, list.p, cnt.p);
  GOD_LAUNCH(seg_merge, (unsigned)num_sms() * 4, kST, 0, st, a, seg_aoff.p, first.p, list.p, cnt.p, tmp.p);
  return GOD_OK;
}

}  // namespace god
