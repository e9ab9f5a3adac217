// Compressed seed index (Sec. 3.1 step 3; Sec. 3.2 filter) and its lookups.
//
// Build: sketch the patterned reference (shift 0), stable-sort the minimizers
// by key (they arrive in position order), cut the sorted array into runs of
// equal keys, drop runs longer than max_occ, and emit
//   keys[U]     kept keys ascending,
//   start[U+1]  offsets of each key's entries,
//   ent[E]      (ref_pos << 1) | z, ascending within a key,
// plus an open-addressing hash table key -> rank at load <= 1/2 (one 64-bit
// word per slot; the rank gives (start, count)).
// The learned index (built in rmi.cu) predicts a key's rank in keys[] instead.
#include <algorithm>

#include "common.cuh"
#include "rmi_device.cuh"

namespace god {
namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(uint64_t n, int per = kThreads) {
  uint64_t b = (n + per - 1) / per;
  return (unsigned)std::min<uint64_t>(std::max<uint64_t>(b, 1), 1u << 30);
}

// Staged sketch records of each warp sub-tile -> keys[] and vals[] =
// (pos << 1) | z at their ordered place (warp per sub-tile).
template <typename V>
__global__ void split_staged(const MinRec* __restrict__ staging, const uint32_t* __restrict__ sub_cnt,
                             const uint64_t* __restrict__ sub_off, uint64_t n_sub, int WT, uint64_t* __restrict__ keys,
                             V* __restrict__ vals) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t sub = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; sub < n_sub; sub += warps) {
    const uint32_t c = sub_cnt[sub];
    const uint64_t o = sub_off[sub];
    const MinRec* src = staging + sub * (uint64_t)WT;
    for (uint32_t i = lane; i < c; i += 32) {
      const uint4 r = __ldcs(reinterpret_cast<const uint4*>(src + i));   // read once
      keys[o + i] = ((uint64_t)r.y << 32) | r.x;
      vals[o + i] = (V)(((uint64_t)r.z << 1) | (r.w & 1u));
    }
  }
}

// The same for the per-segment kernel's staging (segment s's records at
// staging[base[s]]): a warp takes 32 consecutive segments and spreads their
// records over its lanes; a lane finds the segment of its record by a binary
// search over the segments' exclusive counts held one per lane.
template <typename V>
__global__ void split_staged_seg(const MinRec* __restrict__ staging, const uint32_t* __restrict__ cnt,
                                 const uint64_t* __restrict__ off, uint64_t n_seg, const uint64_t* __restrict__ base,
                                 uint64_t* __restrict__ keys, V* __restrict__ vals) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  for (uint64_t grp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / 32; grp * 32 < n_seg; grp += warps) {
    const uint64_t sg = grp * 32 + lane;
    const uint32_t c = sg < n_seg ? cnt[sg] : 0u;
    const uint64_t b = sg < n_seg ? base[sg] : 0;
    uint32_t inc = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, inc, d);
      if (lane >= d) inc += y;
    }
    const uint32_t ex = inc - c;
    const uint32_t tot = __shfl_sync(FULL, inc, 31);
    const uint64_t o0 = off[grp * 32];
    for (uint32_t b0 = 0; b0 < tot; b0 += 32) {   // warp-uniform trip count
      const uint32_t i = b0 + lane;
      int L = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t e = __shfl_sync(FULL, ex, L + step);
        if (e <= i) L += step;
      }
      const uint32_t eL = __shfl_sync(FULL, ex, L);
      const uint64_t bL = __shfl_sync(FULL, b, L);
      if (i < tot) {
        const uint4 r = __ldcs(reinterpret_cast<const uint4*>(staging + bL + (i - eL)));   // read once
        keys[o0 + i] = ((uint64_t)r.y << 32) | r.x;
        vals[o0 + i] = (V)(((uint64_t)r.z << 1) | (r.w & 1u));
      }
    }
  }
}

// Runs of equal keys in the sorted array: the first element of each run
// (its head) finds the run's end by galloping then bisecting, and records
// rv[i] = 1 << 32 | length for a kept run (length <= max_occ), 0 otherwise.
// An exclusive scan of rv then gives every kept run its key rank (high half)
// and its first entry (low half): lengths sum to at most n < 2^32, so the low
// half never carries into the high one.
__global__ void run_heads(const uint64_t* __restrict__ keys, uint64_t n, uint32_t max_occ, uint64_t* __restrict__ rv) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys[i];
    uint64_t v = 0;
    if (i == 0 || keys[i - 1] != key) {
      uint64_t step = 1;
      while (i + step < n && keys[i + step] == key) step <<= 1;
      uint64_t lo = i + (step >> 1), hi = std::min<uint64_t>(i + step, n);   // keys[lo] == key, end in (lo, hi]
      while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        if (keys[mid] == key) lo = mid; else hi = mid;
      }
      const uint64_t len = hi - i;
      if (len <= max_occ) v = (1ULL << 32) | len;
    }
    rv[i] = v;
  }
}

// Kept runs -> keys[U], start[U + 1], ent[E].
template <typename V>
__global__ void emit_runs(const uint64_t* __restrict__ keys, const V* __restrict__ vals, uint64_t n,
                          const uint64_t* __restrict__ rv, const uint64_t* __restrict__ roff,
                          uint64_t* __restrict__ out_keys, uint32_t* __restrict__ out_start,
                          uint64_t* __restrict__ out_ent) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t v = rv[i];
    if (v) {
      const uint64_t o = roff[i];
      const uint32_t u = (uint32_t)(o >> 32), e = (uint32_t)o, len = (uint32_t)v;
      out_keys[u] = keys[i];
      out_start[u] = e;
      for (uint32_t j = 0; j < len; ++j) out_ent[(uint64_t)e + j] = (uint64_t)vals[i + j];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const uint64_t t = roff[n];
    out_start[t >> 32] = (uint32_t)t;
  }
}

// Hash table insert of key rank r (linear probing, one CAS per probe); the
// slot field is start << cb | count (cb > 0) or r. A displacement past the
// field's range sets *overflow (the caller rebuilds a larger table).
__global__ void ht_insert(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ start, uint64_t U,
                          uint64_t* ht, uint32_t lc, uint32_t db, uint32_t rb, uint32_t cb, int* overflow) {
  const uint64_t mask = (1ULL << lc) - 1;
  const uint64_t maxd = (1ULL << db) - 2;
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < U; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys[r];
    const uint64_t h = key & mask, q = key >> lc;
    const uint64_t field = cb ? ((uint64_t)start[r] << cb) | (start[r + 1] - start[r]) : r;
    bool placed = false;
    for (uint64_t d = 0; d <= maxd; ++d) {
      const unsigned long long word = (unsigned long long)((((q << db) | d) << rb) | field);
      unsigned long long* slot = reinterpret_cast<unsigned long long*>(ht + ((h + d) & mask));
      if (atomicCAS(slot, (unsigned long long)kEmptyKey, word) == kEmptyKey) {
        placed = true;
        break;
      }
    }
    if (!placed) atomicExch(overflow, 1);
  }
}

}  // namespace

// ------------------------------------------------------------------ lookups
template <int VIA>
__global__ void __launch_bounds__(kThreads) lookup_kernel(DeviceIndex di, const uint64_t* keys, size_t stride_words,
                                                          uint64_t n, uint64_t* out) {
  __shared__ RmiRoot R;
  if (VIA == 1) {
    if (threadIdx.x == 0) R = *di.root;
    __syncthreads();
  }
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = __ldg(keys + i * stride_words);
    out[i] = VIA == 1 ? rmi_find(di, R, key) : ht_find(di, key);
  }
}

DeviceIndex device_view(const god_index* idx, int via) {
  DeviceIndex d{};
  d.keys = idx->d_keys;
  d.start = idx->d_start;
  d.ent = idx->d_ent;
  d.ht = idx->d_ht;
  d.ht_lc = idx->ht_lc;
  d.ht_db = idx->ht_db;
  d.ht_rb = idx->ht_rb;
  d.ht_cb = idx->ht_cb;
  d.n_keys = idx->n_keys;
  d.leaves = (via == 1 && idx->has_rmi) ? idx->d_leaves : nullptr;
  d.root = (via == 1 && idx->has_rmi) ? idx->d_root : nullptr;
  d.eps_max = idx->params.rmi_eps_max;
  return d;
}

int lookup_keys(const DeviceIndex& di, const uint64_t* keys, size_t key_stride_bytes, uint64_t n, int via,
                uint64_t* out, cudaStream_t st) {
  if (n == 0) return GOD_OK;
  const size_t stride = key_stride_bytes / 8;
  const int sms = num_sms();
  const unsigned grid = (unsigned)std::min<uint64_t>(blocks_for(n), (uint64_t)sms * 16);
  if (via == 1 && di.leaves) {
    GOD_LAUNCH(lookup_kernel<1>, grid, kThreads, 0, st, di, keys, stride, n, out);
    prof_add_work("lookup_kernel<1>", 32.0 * (double)n, (double)n);
  } else {
    GOD_LAUNCH(lookup_kernel<0>, grid, kThreads, 0, st, di, keys, stride, n, out);
    prof_add_work("lookup_kernel<0>", 32.0 * (double)n, (double)n);
  }
  return GOD_OK;
}

// Sort the reference minimizers by key (values: (pos << 1) | z, 32-bit when
// the reference is shorter than 2^31), cut runs, filter, and emit keys,
// offsets and entries. U, E: kept keys and entries.
template <typename V>
int sort_and_emit(god_index* idx, StagedSketch& S, uint64_t n, cudaStream_t st, DBuf<uint64_t>& okeys,
                  DBuf<uint32_t>& ostart, DBuf<uint64_t>& oent, uint64_t* U_out, uint64_t* E_out) {
  DBuf<uint64_t> keys;
  DBuf<V> vals;
  GOD_TRY(keys.alloc(n, st));
  GOD_TRY(vals.alloc(n, st));
  const unsigned g = std::min<unsigned>(blocks_for(n), (unsigned)num_sms() * 32);
  if (n && S.sub_base) {
    const uint64_t blocks =
        std::min<uint64_t>(((S.n_sub + 31) / 32 * 32 + kThreads - 1) / kThreads, (uint64_t)num_sms() * 16);
    GOD_LAUNCH(split_staged_seg<V>, (unsigned)blocks, kThreads, 0, st, S.staging.p, S.sub_cnt.p, S.sub_off.p,
               S.n_sub, S.sub_base, keys.p, vals.p);
  } else if (n) {
    const uint64_t blocks = std::min<uint64_t>((S.n_sub * 32 + kThreads - 1) / kThreads, (uint64_t)num_sms() * 16);
    GOD_LAUNCH(split_staged<V>, (unsigned)blocks, kThreads, 0, st, S.staging.p, S.sub_cnt.p, S.sub_off.p, S.n_sub,
               S.WT, keys.p, vals.p);
  }
  S.staging.release();
  if constexpr (sizeof(V) == 4)
    GOD_TRY(radix_sort_pairs32(keys.p, vals.p, n, 2 * idx->k, st));
  else
    GOD_TRY(radix_sort_pairs(keys.p, vals.p, n, 2 * idx->k, st));

  // runs of equal keys, the filter, and the output arrays
  DBuf<uint64_t> rv, roff;
  GOD_TRY(rv.alloc(n, st));
  GOD_TRY(roff.alloc(n + 1, st));
  if (n) GOD_LAUNCH(run_heads, g, kThreads, 0, st, keys.p, n, idx->max_occ, rv.p);
  GOD_TRY(exclusive_scan_u64(rv.p, roff.p, n, st));
  uint64_t tot = 0;
  GOD_CK(cudaMemcpyAsync(&tot, roff.p + n, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  GOD_TRY(scan_total_ok(tot, "index"));
  const uint64_t U = tot >> 32, E = tot & 0xFFFFFFFFULL;
  GOD_TRY(okeys.alloc(U, st));
  GOD_TRY(ostart.alloc(U + 1, st));
  GOD_TRY(oent.alloc(E, st));
  if (n) {
    GOD_LAUNCH(emit_runs<V>, g, kThreads, 0, st, keys.p, vals.p, n, rv.p, roff.p, okeys.p, ostart.p, oent.p);
  } else {
    GOD_CK(cudaMemsetAsync(ostart.p, 0, sizeof(uint32_t), st));
  }
  *U_out = U;
  *E_out = E;
  return GOD_OK;
}

// ------------------------------------------------------------------ build
// The reference cut into overlapping pieces for the one-thread-per-segment
// sketch kernel: piece i owns the k-mers [i S, (i + 1) S) of the patterned
// reference and holds every window containing one of them (w - 1 k-mers
// before, w - 1 after, and the k - 1 bases of the last k-mer), starting at a
// multiple of the pattern weight x so that its first base has pattern phase 0.
// Its minimizers in the owned range are exactly the whole sequence's there.
// Piece i spans [a_i, b_i) with a_0 = 0, a_i = i S - cw (cw = w - 1 rounded
// up to a multiple of x) and b_i = min(m, (i + 1) S + c) (c = w + k - 2), so
// the virtual offsets (sums of b - a + 1) have a closed form and the pieces
// are generated on the device (no host loop, no descriptor copy).
struct RefPieces {
  uint64_t n = 0, S = 0, cw = 0, c = 0, m = 0, nk = 0, T = 0;
  uint32_t x = 1, p = 1, max_m = 0;
};

__host__ __device__ inline uint64_t ref_voff(const RefPieces& R, uint64_t i) {
  const uint64_t t = i < R.T ? i : R.T;   // pieces before i that end inside the reference
  const uint64_t sb = R.S * t * (t + 1) / 2 + R.c * t + (i - t) * R.m;
  const uint64_t sa = i ? R.S * i * (i - 1) / 2 - R.cw * (i - 1) : 0;
  return sb - sa + i;
}

__global__ void make_ref_pieces(RefPieces R, SegDesc* __restrict__ segs, uint64_t* __restrict__ voff,
                                uint32_t* __restrict__ own) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= R.n; i += (uint64_t)gridDim.x * blockDim.x) {
    voff[i] = ref_voff(R, i);
    if (i == R.n) continue;
    const uint64_t lo = i * R.S, hi = lo + R.S < R.nk ? lo + R.S : R.nk;
    const uint64_t a = i ? lo - R.cw : 0;
    const uint64_t b = lo + R.S + R.c < R.m ? lo + R.S + R.c : R.m;
    segs[i] = SegDesc{0, (uint32_t)(b - a), 0, (uint32_t)((uint64_t)R.p * (a / R.x)), 0};
    own[2 * i] = (uint32_t)(lo - a);
    own[2 * i + 1] = (uint32_t)(hi - a);
  }
}

bool ref_pieces(const PatternInfo& P, uint64_t m, int k, int w, RefPieces* R) {
  const uint64_t x = (uint64_t)P.x;
  const uint64_t cw = ((uint64_t)(w - 1) + x - 1) / x * x, c = (uint64_t)(w + k - 2);
  if (m < (uint64_t)k) return false;
  // piece length (patterned bases): short enough for every SM to hold its
  // warps two rounds over (a warp takes 32 pieces; about 24 warps per SM),
  // at least 256 (the halo's share of the work), at most 2048
  const uint64_t lanes = (uint64_t)num_sms() * 24 * 32 * 2;
  const uint64_t span = std::min<uint64_t>(2048, std::max<uint64_t>(256, m / lanes + cw + c));
  if (span <= cw + c + x) return false;
  R->S = (span - cw - c) / x * x;
  R->cw = cw;
  R->c = c;
  R->m = m;
  R->nk = m - k + 1;
  R->n = (R->nk + R->S - 1) / R->S;
  R->T = m >= c ? (m - c) / R->S : 0;
  R->x = (uint32_t)x;
  R->p = (uint32_t)P.p;
  R->max_m = (uint32_t)(R->S + cw + c);
  return R->n >= 1024 && R->n < (1ull << 31);   // long references only
}

int build_index_device(god_index* idx, const uint8_t* d_ref, uint64_t len, cudaStream_t st) {
  const PatternInfo& P = idx->pat;
  const uint64_t m = patterned_len(P, len, 0);
  idx->n_min = idx->n_keys = idx->n_ent = 0;
  DBuf<SegDesc> seg;
  DBuf<uint64_t> voff;
  DBuf<uint32_t> own;
  SketchJob job{};
  job.bytes = d_ref;
  job.k = idx->k;
  job.w = idx->w;
  job.pat = P;
  job.tune = idx->params.tune;
  RefPieces R;
  StagedSketch S;
  uint64_t n = 0;
  // pieces only for a device-resident reference: 32 pieces span more bytes
  // than a warp stages, and the tile kernel's coalesced gather reads
  // page-locked host bytes better than one lane per piece
  bool pieces = is_device_ptr(d_ref) && ref_pieces(P, m, idx->k, idx->w, &R);
  if (pieces) {
    job.n_seg = (uint32_t)R.n;
    job.V = ref_voff(R, R.n);
    job.max_m = R.max_m;
    pieces = sketch_segments_ok(job);
  }
  if (pieces) {
    const uint64_t np = R.n;
    GOD_TRY(seg.alloc(np, st));
    GOD_TRY(voff.alloc(np + 1, st));
    GOD_TRY(own.alloc(2 * np, st));
    GOD_LAUNCH(make_ref_pieces, (unsigned)std::min<uint64_t>((np + kThreads) / kThreads, (uint64_t)num_sms() * 8),
               kThreads, 0, st, R, seg.p, voff.p, own.p);
    job.segs = seg.p;
    job.seg_voff = voff.p;
    job.own = own.p;
    GOD_TRY(run_sketch_segments(job, st, S));
    GOD_CK(cudaMemcpyAsync(&n, S.sub_off.p + S.n_sub, 8, cudaMemcpyDeviceToHost, st));
    GOD_CK(cudaStreamSynchronize(st));
    GOD_TRY(scan_total_ok(n, "index"));
    S.total = n;
  } else {
    GOD_TRY(seg.alloc(1, st));
    GOD_TRY(voff.alloc(2, st));
    SegDesc hs{0, (uint32_t)m, 0, 0, 0};
    uint64_t hv[2] = {0, m + 1};
    GOD_CK(cudaMemcpyAsync(seg.p, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    GOD_CK(cudaMemcpyAsync(voff.p, hv, sizeof(hv), cudaMemcpyHostToDevice, st));
    job.segs = seg.p;
    job.seg_voff = voff.p;
    job.n_seg = 1;
    job.V = m + 1;
    job.own = nullptr;
    job.max_m = 0;
    GOD_TRY(run_sketch_staged(job, st, S, nullptr));
    n = S.total;
  }
  idx->n_min = n;

  DBuf<uint64_t> okeys, oent;
  DBuf<uint32_t> ostart;
  uint64_t U = 0, E = 0;
  if (len < (1ULL << 31))
    GOD_TRY(sort_and_emit<uint32_t>(idx, S, n, st, okeys, ostart, oent, &U, &E));
  else
    GOD_TRY(sort_and_emit<uint64_t>(idx, S, n, st, okeys, ostart, oent, &U, &E));
  // hash table at load <= 1/2; the slot word splits 64 bits into the quotient
  // (2k - lc bits), the field (rb bits) and the displacement (the rest). The
  // field is the key's (start, count) when that leaves at least 8
  // displacement bits, else its rank (then >= 9 displacement bits for k <= 28
  // since 2^lc >= 2U)
  uint32_t rank_bits = 1;
  while (rank_bits < 63 && (1ULL << rank_bits) < U) ++rank_bits;
  uint32_t start_bits = 1, count_bits = 1;
  while (start_bits < 40 && (1ULL << start_bits) < E) ++start_bits;
  while (count_bits < 32 && (1ULL << count_bits) <= std::min<uint64_t>(idx->max_occ, E)) ++count_bits;
  uint32_t lc = 4;
  while ((1ULL << lc) < 2 * U) ++lc;
  DBuf<uint64_t> ht;
  DBuf<int> ovf;
  GOD_TRY(ovf.alloc(1, st));
  for (;; ++lc) {
    const uint32_t qb = 2 * idx->k > (int)lc ? 2 * idx->k - lc : 0;
    const bool payload = qb + start_bits + count_bits + 8 <= 64;
    const uint32_t rb = payload ? start_bits + count_bits : rank_bits;
    const uint32_t cb = payload ? count_bits : 0;
    const uint32_t db = 64 - qb - rb;
    if (qb + rb > 62 || lc > 40) {
      set_error("index: hash table does not fit");
      return GOD_EINVAL;
    }
    const uint64_t cap = 1ULL << lc;
    GOD_TRY(ht.alloc(cap, st));
    GOD_CK(cudaMemsetAsync(ht.p, 0xFF, cap * sizeof(uint64_t), st));
    GOD_CK(cudaMemsetAsync(ovf.p, 0, sizeof(int), st));
    if (U) GOD_LAUNCH(ht_insert, std::min<unsigned>(blocks_for(U), (unsigned)num_sms() * 32), kThreads, 0, st,
                      okeys.p, ostart.p, U, ht.p, lc, db, rb, cb, ovf.p);
    int h_ovf = 0;
    GOD_CK(cudaMemcpyAsync(&h_ovf, ovf.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GOD_CK(cudaStreamSynchronize(st));
    if (!h_ovf) {
      idx->ht_lc = lc;
      idx->ht_db = db;
      idx->ht_rb = rb;
      idx->ht_cb = cb;
      idx->ht_cap = cap;
      break;
    }
    ht.release();
  }
  idx->n_keys = U;
  idx->n_ent = E;
  idx->d_keys = okeys.take();
  idx->d_start = ostart.take();
  idx->d_ent = oent.take();
  idx->d_ht = ht.take();
  idx->device_bytes = U * 8 + (U + 1) * 4 + E * 8 + idx->ht_cap * 8;
  return GOD_OK;
}

}  // namespace god
