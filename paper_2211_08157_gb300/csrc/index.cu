// Compressed seed index (Sec. 3.1 step 3; Sec. 3.2 filter) and its lookups.
//
// Build: sketch the patterned reference (shift 0), stable-sort the minimizers
// by key (they arrive in position order), cut the sorted array into runs of
// equal keys, drop runs longer than max_occ, and emit
//   keys[U]     kept keys ascending,
//   start[U+1]  offsets of each key's entries,
//   ent[E]      (ref_pos << 1) | z, ascending within a key,
// plus an open-addressing hash table key -> (start, count) at load <= 1/2.
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

__global__ void split_records(const MinRec* rec, uint64_t n, uint64_t* keys, uint64_t* vals) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const MinRec r = rec[i];
    keys[i] = r.key;
    vals[i] = ((uint64_t)r.pos << 1) | (r.segz & 1u);
  }
}

__global__ void mark_heads(const uint64_t* keys, uint64_t n, uint32_t* head) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

// run_excl[i] = heads before i (n + 1 entries). Heads record their run start.
__global__ void run_starts(const uint32_t* head, const uint64_t* run_excl, uint64_t n, uint64_t* run_start,
                           uint64_t n_runs) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (head[i]) run_start[run_excl[i]] = i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) run_start[n_runs] = n;
}

__global__ void run_keep(const uint64_t* run_start, uint64_t n_runs, uint32_t max_occ, uint32_t* kept,
                         uint64_t* kept_len) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n_runs; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t len = run_start[r + 1] - run_start[r];
    const bool k = len <= max_occ;
    kept[r] = k;
    kept_len[r] = k ? len : 0;
  }
}

__global__ void emit_keys(const uint64_t* keys, const uint64_t* run_start, const uint32_t* kept,
                          const uint64_t* kept_rank, const uint64_t* ent_off, uint64_t n_runs, uint64_t* out_keys,
                          uint32_t* out_start) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n_runs; r += (uint64_t)gridDim.x * blockDim.x) {
    if (kept[r]) {
      out_keys[kept_rank[r]] = keys[run_start[r]];
      out_start[kept_rank[r]] = (uint32_t)ent_off[r];
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out_start[kept_rank[n_runs]] = (uint32_t)ent_off[n_runs];
}

__global__ void emit_entries(const uint64_t* vals, const uint64_t* run_excl, const uint64_t* run_start,
                             const uint32_t* kept, const uint64_t* ent_off, uint64_t n, uint64_t* out_ent) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = run_excl[i + 1] - 1;  // heads in [0, i] minus one
    if (kept[r]) out_ent[ent_off[r] + (i - run_start[r])] = vals[i];
  }
}

__global__ void ht_insert(const uint64_t* keys, const uint32_t* start, uint64_t n, ulonglong2* ht, uint64_t mask) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys[r];
    const uint64_t payload = (uint64_t)start[r] | ((uint64_t)(start[r + 1] - start[r]) << 32);
    uint64_t slot = key & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      unsigned long long* kp = reinterpret_cast<unsigned long long*>(&ht[slot].x);
      const unsigned long long prev = atomicCAS(kp, (unsigned long long)kEmptyKey, (unsigned long long)key);
      if (prev == kEmptyKey) {
        ht[slot].y = payload;
        break;
      }
      slot = (slot + 1) & mask;
    }
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
    out[i] = VIA == 1 ? rmi_find(di, R, key) : ht_find(di.ht, di.ht_mask, key);
  }
}

DeviceIndex device_view(const god_index* idx, int via) {
  DeviceIndex d{};
  d.keys = idx->d_keys;
  d.start = idx->d_start;
  d.ent = idx->d_ent;
  d.ht = idx->d_ht;
  d.ht_mask = idx->ht_cap - 1;
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

// ------------------------------------------------------------------ build
int build_index_device(god_index* idx, const uint8_t* d_ref, uint64_t len, cudaStream_t st) {
  const PatternInfo& P = idx->pat;
  const uint64_t m = patterned_len(P, len, 0);
  idx->n_min = idx->n_keys = idx->n_ent = 0;
  DBuf<SegDesc> seg;
  DBuf<uint64_t> voff;
  GOD_TRY(seg.alloc(1, st));
  GOD_TRY(voff.alloc(2, st));
  SegDesc hs{0, (uint32_t)m, 0, 0, 0};
  uint64_t hv[2] = {0, m + 1};
  GOD_CK(cudaMemcpyAsync(seg.p, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
  GOD_CK(cudaMemcpyAsync(voff.p, hv, sizeof(hv), cudaMemcpyHostToDevice, st));

  SketchJob job{};
  job.bytes = d_ref;
  job.segs = seg.p;
  job.seg_voff = voff.p;
  job.n_seg = 1;
  job.V = m + 1;
  job.k = idx->k;
  job.w = idx->w;
  job.pat = P;
  job.tune = idx->params.tune;
  DBuf<MinRec> rec;
  uint64_t total = 0;
  GOD_TRY(run_sketch(job, st, rec, &total, nullptr));
  const uint64_t n = total;
  idx->n_min = n;

  DBuf<uint64_t> keys, vals;
  GOD_TRY(keys.alloc(n, st));
  GOD_TRY(vals.alloc(n, st));
  const unsigned g = std::min<unsigned>(blocks_for(n), (unsigned)num_sms() * 32);
  if (n) GOD_LAUNCH(split_records, g, kThreads, 0, st, rec.p, n, keys.p, vals.p);
  rec.release();
  GOD_TRY(radix_sort_pairs(keys.p, vals.p, n, 2 * idx->k, st));

  // runs of equal keys
  DBuf<uint32_t> head;
  DBuf<uint64_t> run_excl;
  GOD_TRY(head.alloc(n, st));
  GOD_TRY(run_excl.alloc(n + 1, st));
  if (n) GOD_LAUNCH(mark_heads, g, kThreads, 0, st, keys.p, n, head.p);
  GOD_TRY(exclusive_scan_u32(head.p, run_excl.p, n, st));
  uint64_t n_runs = 0;
  GOD_CK(cudaMemcpyAsync(&n_runs, run_excl.p + n, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  DBuf<uint64_t> run_start, kept_len, kept_rank, ent_off;
  DBuf<uint32_t> kept;
  GOD_TRY(run_start.alloc(n_runs + 1, st));
  GOD_TRY(kept.alloc(n_runs, st));
  GOD_TRY(kept_len.alloc(n_runs, st));
  GOD_TRY(kept_rank.alloc(n_runs + 1, st));
  GOD_TRY(ent_off.alloc(n_runs + 1, st));
  const unsigned gr = std::min<unsigned>(blocks_for(n_runs), (unsigned)num_sms() * 32);
  GOD_LAUNCH(run_starts, g, kThreads, 0, st, head.p, run_excl.p, n, run_start.p, n_runs);
  if (n_runs) GOD_LAUNCH(run_keep, gr, kThreads, 0, st, run_start.p, n_runs, idx->max_occ, kept.p, kept_len.p);
  GOD_TRY(exclusive_scan_u32(kept.p, kept_rank.p, n_runs, st));
  GOD_TRY(exclusive_scan_u64(kept_len.p, ent_off.p, n_runs, st));
  uint64_t sizes[2] = {0, 0};
  GOD_CK(cudaMemcpyAsync(&sizes[0], kept_rank.p + n_runs, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaMemcpyAsync(&sizes[1], ent_off.p + n_runs, 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  const uint64_t U = sizes[0], E = sizes[1];
  if (E >= (1ULL << 32)) {
    set_error("index: more than 2^32 entries");
    return GOD_EINVAL;
  }
  DBuf<uint64_t> okeys, oent;
  DBuf<uint32_t> ostart;
  GOD_TRY(okeys.alloc(U, st));
  GOD_TRY(ostart.alloc(U + 1, st));
  GOD_TRY(oent.alloc(E, st));
  GOD_LAUNCH(emit_keys, gr, kThreads, 0, st, keys.p, run_start.p, kept.p, kept_rank.p, ent_off.p, n_runs, okeys.p,
             ostart.p);
  if (n) GOD_LAUNCH(emit_entries, g, kThreads, 0, st, vals.p, run_excl.p, run_start.p, kept.p, ent_off.p, n, oent.p);

  // hash table at load <= 1/2
  uint64_t cap_ht = 16;
  while (cap_ht < 2 * U) cap_ht <<= 1;
  DBuf<ulonglong2> ht;
  GOD_TRY(ht.alloc(cap_ht, st));
  GOD_CK(cudaMemsetAsync(ht.p, 0xFF, cap_ht * sizeof(ulonglong2), st));
  if (U) GOD_LAUNCH(ht_insert, std::min<unsigned>(blocks_for(U), (unsigned)num_sms() * 32), kThreads, 0, st,
                    okeys.p, ostart.p, U, ht.p, cap_ht - 1);
  GOD_CK(cudaStreamSynchronize(st));
  idx->n_keys = U;
  idx->n_ent = E;
  idx->d_keys = okeys.take();
  idx->d_start = ostart.take();
  idx->d_ent = oent.take();
  idx->d_ht = ht.take();
  idx->ht_cap = cap_ht;
  idx->device_bytes = U * 8 + (U + 1) * 4 + E * 8 + cap_ht * 16;
  return GOD_OK;
}

}  // namespace god
