// Continuous-batching seeding server over one resident index.
//
// Requests (read batches) are queued on submit. Each of `slots` worker threads
// owns a CUDA stream and pinned staging buffers; whenever it is free it admits
// the oldest waiting request plus as many further waiting requests as fit in
// max_batch_bases, provided the batch's device-memory estimate fits in what
// the budget has left. The merged batch runs through the same batched seeding
// pass as god_seed (one sketch launch over all of its reads), then the sorted
// anchor list is cut back into per-request arrays by read range (anchors are
// sorted by read, so each request owns one contiguous run) without a copy: the
// batch's anchors land in one page-locked buffer whose slices are the
// requests' results. Slots run
// concurrently, so requests that arrive while others are on the GPU overlap
// with them. Integer results do not depend on how requests were merged.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Arena;

struct Request {
  uint64_t id;
  const uint8_t* reads = nullptr;   // the caller's bytes (valid until its wait returns)
  std::vector<uint64_t> offs;       // n + 1, rebased to 0
  uint32_t n;
  uint64_t bases;
  Clock::time_point t_submit, t_done;
  bool done = false;
  bool merged = false;
  int rc = GOD_OK;
  god_anchor* result = nullptr;   // a slice of `arena`, or malloc'ed when empty
  Arena* arena = nullptr;
  uint64_t n_result = 0;
};

// Page-locked host memory cache shared by every server of the process.
// Pinning fresh memory (cudaMallocHost) runs at a few GB/s and holds the
// driver's lock meanwhile, stalling the other slots' CUDA calls; measured on
// the serving stream it took a third of the slots' time. So buffers go back
// to this cache rather than to the system, and later batches (and later
// servers) take them again. Blocks are sized with headroom so that they fit
// more batches; a block is taken only for needs of at least a quarter of its
// size; free blocks beyond kPinCacheCap bytes are released.
constexpr uint64_t kPinCacheCap = 16ull << 30;
struct PinCache {
  std::mutex mu;
  std::multimap<uint64_t, void*> free_blocks;   // size -> block
  uint64_t cached = 0;
};
PinCache& pin_cache() {
  static PinCache* c = new PinCache();   // never destroyed: slices may outlive static destruction order
  return *c;
}

void* pinned_take(uint64_t need, uint64_t* got) {
  PinCache& C = pin_cache();
  {
    std::lock_guard<std::mutex> lk(C.mu);
    auto it = C.free_blocks.lower_bound(need);
    if (it != C.free_blocks.end() && it->first / 4 <= need) {
      void* p = it->second;
      *got = it->first;
      C.cached -= it->first;
      C.free_blocks.erase(it);
      return p;
    }
  }
  // headroom: the next power of two at or above 1.25 x need (at least 4 MiB)
  uint64_t sz = 4ull << 20;
  while (sz < need + need / 4) sz <<= 1;
  void* p = nullptr;
  if (cudaMallocHost(&p, sz) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  *got = sz;
  return p;
}

void pinned_give(void* p, uint64_t size) {
  if (!p) return;
  PinCache& C = pin_cache();
  {
    std::lock_guard<std::mutex> lk(C.mu);
    if (C.cached + size <= kPinCacheCap) {
      C.free_blocks.emplace(size, p);
      C.cached += size;
      return;
    }
  }
  cudaFreeHost(p);
}

// Page-locked buffer holding one batch's anchors; every request of the batch
// gets its result as a slice of it (no per-request copy), and the buffer goes
// back to the cache when the last slice has been freed (god_free), also after
// the server is gone.
struct Arena {
  god_anchor* p = nullptr;
  uint64_t bytes = 0;
  std::atomic<int> refs{0};     // live slices
};

void arena_release(void* ctx) {
  Arena* a = static_cast<Arena*>(ctx);
  if (a->refs.fetch_sub(1) == 1) {
    pinned_give(a->p, a->bytes);
    delete a;
  }
}

// A buffer for `need` anchors.
Arena* arena_take(uint64_t need) {
  Arena* a = new Arena();
  uint64_t got = 0;
  a->p = static_cast<god_anchor*>(pinned_take(std::max<uint64_t>(need, 1) * sizeof(god_anchor), &got));
  if (!a->p) {
    delete a;
    return nullptr;
  }
  a->bytes = got;
  return a;
}

// memcpy of a batch's request bytes into the pinned staging buffer, split over
// a few threads when it is large (one thread copies well below the memory
// bandwidth of the host).
void gather_bytes(const std::vector<std::pair<const uint8_t*, uint64_t>>& parts, uint8_t* dst) {
  uint64_t total = 0;
  for (auto& pr : parts) total += pr.second;
  const int nt = total >= (16ull << 20) ? 4 : 1;
  auto copy_range = [&](uint64_t lo, uint64_t hi) {   // byte range [lo, hi) of the concatenation
    uint64_t at = 0;
    for (auto& pr : parts) {
      const uint64_t a = std::max(lo, at), b = std::min(hi, at + pr.second);
      if (a < b) memcpy(dst + a, pr.first + (a - at), b - a);
      at += pr.second;
      if (at >= hi) break;
    }
  };
  if (nt == 1) {
    copy_range(0, total);
    return;
  }
  std::vector<std::thread> th;
  for (int i = 1; i < nt; ++i) th.emplace_back(copy_range, total * i / nt, total * (i + 1) / nt);
  copy_range(0, total / nt);
  for (auto& t : th) t.join();
}

// Device bytes a batch may hold at its peak: input, segment tables, minimizer
// records, lookups and the anchor output (estimated at 2 anchors per kept
// minimizer), with a safety factor.
uint64_t batch_bytes_estimate(const god_index* idx, uint64_t bases, uint64_t n) {
  const double mins = (double)bases * idx->pat.x / idx->pat.p * 2.0 / (idx->w + 1) * idx->pat.p;
  const double b = (double)bases * 1.0 + (double)n * (8 + 48.0 * idx->pat.p) + mins * (16 + 8 + 8) +
                   mins * 2.0 * 16 * 2;
  return (uint64_t)(b * 1.5) + (16ull << 20);
}

// bounds[j] = first anchor of request j (anchors sorted by batch read id;
// request j owns batch reads [first[j], first[j + 1])), bounds[m] = n.
__global__ void request_bounds(const god_anchor* __restrict__ a, uint64_t n, const uint32_t* __restrict__ first,
                               uint32_t m, uint64_t* __restrict__ bounds) {
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= m; j += gridDim.x * blockDim.x) {
    if (j == m) {
      bounds[j] = n;
      continue;
    }
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (a[mid].read_id < first[j]) lo = mid + 1; else hi = mid;
    }
    bounds[j] = lo;
  }
}

// Read ids back to each request's own numbering.
__global__ void rebase_read_ids(god_anchor* __restrict__ a, uint64_t n, const uint32_t* __restrict__ first,
                                uint32_t m) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t r = a[i].read_id;
    uint32_t lo = 0, hi = m;                   // largest j with first[j] <= r
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (first[mid] <= r) lo = mid; else hi = mid;
    }
    a[i].read_id = r - first[lo];
  }
}

int split_on_device(god_anchor* d_out, uint64_t total, const uint32_t* d_first, uint32_t m, uint64_t* d_bounds,
                    cudaStream_t st) {
  GOD_LAUNCH(request_bounds, (m + 128) / 128, 128, 0, st, d_out, total, d_first, m, d_bounds);
  if (total)
    GOD_LAUNCH(rebase_read_ids, (unsigned)std::min<uint64_t>((total + 255) / 256, 4096), 256, 0, st, d_out, total,
               d_first, m);
  return GOD_OK;
}

}  // namespace

struct god_server {
  const god_index* idx = nullptr;
  god_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<std::thread> workers;
  uint64_t next_id = 1;
  uint64_t mem_in_use = 0;
  uint64_t inflight = 0;
  bool stop = false;
  god_server_stats st{};
};

namespace {

void worker_main(god_server* S, int slot) {
  cudaSetDevice(S->idx->device);
  cudaStream_t stream;
  cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  uint8_t* h_reads = nullptr;
  uint64_t* h_offs = nullptr;
  uint64_t cap_reads = 0, cap_offs = 0;   // bytes
  (void)slot;
  while (true) {
    std::vector<Request*> batch;
    uint64_t est = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      while (true) {
        if (S->stop) break;
        if (!S->queue.empty()) {
          // admission: oldest request first, then merge while it fits
          uint64_t bases = 0, reads = 0;
          size_t take = 0;
          for (size_t i = 0; i < S->queue.size(); ++i) {
            Request* r = S->queue[i];
            if (take > 0 && bases + r->bases > S->cfg.max_batch_bases) break;
            bases += r->bases;
            reads += r->n;
            ++take;
          }
          est = batch_bytes_estimate(S->idx, bases, reads);
          // shrink the batch until it fits the remaining budget
          while (take > 1 && S->mem_in_use + est > S->cfg.mem_budget) {
            --take;
            bases -= S->queue[take]->bases;
            reads -= S->queue[take]->n;
            est = batch_bytes_estimate(S->idx, bases, reads);
          }
          if (S->mem_in_use + est <= S->cfg.mem_budget) {
            for (size_t i = 0; i < take; ++i) {
              batch.push_back(S->queue.front());
              S->queue.pop_front();
            }
            S->mem_in_use += est;
            S->inflight++;
            S->st.batches++;
            S->st.max_inflight_batches = std::max(S->st.max_inflight_batches, S->inflight);
            if (batch.size() > 1) S->st.merged_requests += batch.size();
            break;
          }
          if (S->inflight == 0) {
            // a single request larger than the whole budget: reject it
            Request* r = S->queue.front();
            S->queue.pop_front();
            r->rc = GOD_ENOMEM;
            r->done = true;
            r->t_done = Clock::now();
            S->st.rejected++;
            S->st.completed++;
            S->cv_done.notify_all();
            continue;
          }
        }
        S->cv_work.wait(lk);
      }
      if (S->stop && batch.empty()) break;
    }
    // ---- concatenate the batch into pinned staging
    auto secs = [](Clock::time_point a, Clock::time_point b) { return std::chrono::duration<double>(b - a).count(); };
    double t_alloc = 0.0;
    const auto t0 = Clock::now();
    uint64_t bases = 0, n = 0;
    for (Request* r : batch) { bases += r->bases; n += r->n; }
    int rc = GOD_OK;
    if (bases > cap_reads) {
      const auto a0 = Clock::now();
      pinned_give(h_reads, cap_reads);
      h_reads = static_cast<uint8_t*>(pinned_take(bases, &cap_reads));
      if (!h_reads) { cap_reads = 0; rc = GOD_ENOMEM; }
      t_alloc += secs(a0, Clock::now());
    }
    if (rc == GOD_OK && (n + 1) * 8 > cap_offs) {
      const auto a0 = Clock::now();
      pinned_give(h_offs, cap_offs);
      h_offs = static_cast<uint64_t*>(pinned_take((n + 1) * 8, &cap_offs));
      if (!h_offs) { cap_offs = 0; rc = GOD_ENOMEM; }
      t_alloc += secs(a0, Clock::now());
    }
    std::vector<uint64_t> first_read;
    if (rc == GOD_OK) {
      uint64_t bo = 0, ro = 0;
      std::vector<std::pair<const uint8_t*, uint64_t>> parts;
      for (Request* r : batch) {
        parts.emplace_back(r->reads, r->bases);
        for (uint32_t i = 0; i < r->n; ++i) h_offs[ro + i] = bo + r->offs[i];
        first_read.push_back(ro);
        bo += r->bases;
        ro += r->n;
      }
      h_offs[ro] = bo;
      gather_bytes(parts, h_reads);
    }
    const auto t1 = Clock::now();
    // ---- device pass
    god::DBuf<uint8_t> d_reads;
    god::DBuf<uint64_t> d_offs;
    god_anchor* d_out = nullptr;
    uint64_t total = 0;
    if (rc == GOD_OK) rc = d_reads.alloc(bases, stream);
    if (rc == GOD_OK) rc = d_offs.alloc(n + 1, stream);
    if (rc == GOD_OK && bases) rc = cudaMemcpyAsync(d_reads.p, h_reads, bases, cudaMemcpyHostToDevice, stream) ? GOD_ECUDA : GOD_OK;
    if (rc == GOD_OK) rc = cudaMemcpyAsync(d_offs.p, h_offs, (n + 1) * 8, cudaMemcpyHostToDevice, stream) ? GOD_ECUDA : GOD_OK;
    if (rc == GOD_OK) {
      god_seed_opts o;
      god_seed_opts_init(&o);
      o.stream = stream;
      rc = god::seed_device(S->idx, d_reads.p, d_offs.p, (uint32_t)n, bases, o, stream, &d_out, &total, nullptr, 0,
                            true);
    }
    const auto t2 = Clock::now();
    Arena* arena = nullptr;
    if (rc == GOD_OK && total) {
      arena = arena_take(total);
      if (!arena) rc = GOD_ENOMEM;
    }
    const auto t3 = Clock::now();
    t_alloc += secs(t2, t3);
    // request boundaries and per-request read ids on the device, so the
    // split below is one copy per request
    const uint32_t m = (uint32_t)batch.size();
    std::vector<uint64_t> bounds(m + 1, 0);
    god::DBuf<uint32_t> d_first;
    god::DBuf<uint64_t> d_bounds;
    if (rc == GOD_OK) rc = d_first.alloc(m, stream);
    if (rc == GOD_OK) rc = d_bounds.alloc(m + 1, stream);
    std::vector<uint32_t> first32(first_read.begin(), first_read.end());
    if (rc == GOD_OK)
      rc = cudaMemcpyAsync(d_first.p, first32.data(), m * 4, cudaMemcpyHostToDevice, stream) ? GOD_ECUDA : GOD_OK;
    if (rc == GOD_OK) rc = split_on_device(d_out, total, d_first.p, m, d_bounds.p, stream);
    if (rc == GOD_OK)
      rc = cudaMemcpyAsync(bounds.data(), d_bounds.p, (m + 1) * 8, cudaMemcpyDeviceToHost, stream) ? GOD_ECUDA : GOD_OK;
    if (rc == GOD_OK && total)
      rc = cudaMemcpyAsync(arena->p, d_out, total * sizeof(god_anchor), cudaMemcpyDeviceToHost, stream) ? GOD_ECUDA
                                                                                                     : GOD_OK;
    if (d_out) god::dfree(d_out, stream);
    d_first.release();
    d_bounds.release();
    d_reads.release();
    d_offs.release();
    if (cudaStreamSynchronize(stream) != cudaSuccess && rc == GOD_OK) rc = GOD_ECUDA;
    const auto t4 = Clock::now();
    // ---- split per request: slices of the arena (an empty result gets a
    // small host array of its own, so that every result pointer is distinct)
    int slices = 0;
    for (size_t bi = 0; bi < batch.size(); ++bi) {
      Request* r = batch[bi];
      r->rc = rc;
      if (rc == GOD_OK) {
        r->n_result = bounds[bi + 1] - bounds[bi];
        if (r->n_result) {
          r->result = arena->p + bounds[bi];
          r->arena = arena;
          ++slices;
        } else {
          r->result = (god_anchor*)malloc(sizeof(god_anchor));
          if (!r->result) r->rc = GOD_ENOMEM;
        }
      }
      r->merged = batch.size() > 1;
    }
    if (arena) {
      if (slices == 0) {
        pinned_give(arena->p, arena->bytes);
        delete arena;
      } else {
        arena->refs.store(slices);
      }
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const auto now = Clock::now();
      for (Request* r : batch) {
        r->done = true;
        r->t_done = now;
        S->st.completed++;
      }
      S->mem_in_use -= est;
      S->inflight--;
      S->st.gather_s += secs(t0, t1) - (t_alloc - secs(t2, t3));
      S->st.pin_alloc_s += t_alloc;
      S->st.device_s += secs(t1, t2);
      S->st.copy_back_s += secs(t3, t4);
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
  pinned_give(h_reads, cap_reads);
  pinned_give(h_offs, cap_offs);
  cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

void god_server_config_init(god_server_config* c) {
  if (!c) return;
  c->slots = 4;
  c->mem_budget = 0;
  c->max_batch_bases = 64ull << 20;
}

int god_server_create(const god_index* idx, const god_server_config* cfg, god_server** out) {
  if (!idx || !out) return GOD_EINVAL;
  god_server* S = new god_server();
  S->idx = idx;
  god_server_config_init(&S->cfg);
  if (cfg) S->cfg = *cfg;
  if (S->cfg.slots < 1) S->cfg.slots = 1;
  if (S->cfg.slots > 32) S->cfg.slots = 32;
  if (S->cfg.max_batch_bases == 0) S->cfg.max_batch_bases = 64ull << 20;
  if (S->cfg.mem_budget == 0) {
    size_t fr = 0, tot = 0;
    cudaSetDevice(idx->device);
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      delete S;
      return god::cuda_fail(cudaGetLastError(), "cudaMemGetInfo", __FILE__, __LINE__);
    }
    S->cfg.mem_budget = (uint64_t)(fr * 0.8);
  }
  for (int i = 0; i < S->cfg.slots; ++i) S->workers.emplace_back(worker_main, S, i);
  *out = S;
  return GOD_OK;
}

int god_server_submit(god_server* S, const uint8_t* reads, const uint64_t* offsets, uint32_t n, uint64_t* request_id) {
  if (!S || !request_id || (n && (!reads || !offsets))) return GOD_EINVAL;
  Request* r = new Request();
  r->n = n;
  const uint64_t b0 = n ? offsets[0] : 0;
  r->offs.resize((size_t)n + 1);
  for (uint32_t i = 0; i <= n; ++i) {
    if (i && (offsets[i] < offsets[i - 1] || offsets[i] - offsets[i - 1] >= (1ull << 31))) {
      delete r;
      god::set_error("offsets must be non-decreasing and each read < 2^31 bytes");
      return GOD_EINVAL;
    }
    r->offs[i] = offsets[i] - b0;
  }
  r->bases = n ? offsets[n] - b0 : 0;
  r->reads = reads + b0;
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    S->st.submitted++;
  }
  S->cv_work.notify_one();
  *request_id = r->id;
  return GOD_OK;
}

int god_server_wait(god_server* S, uint64_t id, int timeout_ms, god_anchor** anchors, uint64_t* n_anchors,
                    double* latency_s) {
  if (!S || !anchors || !n_anchors) return GOD_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return GOD_EINVAL;
  Request* r = it->second;
  if (timeout_ms < 0) S->cv_done.wait(lk, [&] { return r->done; });
  else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; })) return GOD_EBUSY;
  S->reqs.erase(it);
  lk.unlock();
  const int rc = r->rc;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  *anchors = nullptr;
  *n_anchors = 0;
  if (rc == GOD_OK) {
    *anchors = r->result;
    *n_anchors = r->n_result;
    if (r->arena) god::register_slice(r->result, arena_release, r->arena);
    else god::register_host_array(r->result);
  } else if (r->arena) {
    arena_release(r->arena);
  } else if (r->result) {
    free(r->result);
  }
  delete r;
  return rc;
}

int god_server_get_stats(god_server* S, god_server_stats* st) {
  if (!S || !st) return GOD_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->st;
  return GOD_OK;
}

int god_server_destroy(god_server* S) {
  if (!S) return GOD_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& kv : S->reqs) {
    if (kv.second->arena) arena_release(kv.second->arena);
    else if (kv.second->result) free(kv.second->result);
    delete kv.second;
  }
  // arenas with live slices outlive the server; the last slice returns them
  delete S;
  return GOD_OK;
}

}  // extern "C"
