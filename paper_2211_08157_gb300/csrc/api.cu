// C ABI entry points of libgod (declared in include/god.h): argument checks,
// host/device marshalling, ownership registry, and the calls into the
// index / seeding / sketch pipelines.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace god {

std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_prof_on{0};
std::atomic<int> g_graphs_on{1};
static thread_local std::string t_last_error;

// ---- opt-in kernel timing
struct ProfPending {
  const char* name;
  cudaEvent_t a, b;
  cudaStream_t st;
};
// Optional timeline: every timed launch as (kernel, stream, start, end) in ms
// after the base event recorded when timing was switched on or reset.
struct ProfSpan {
  const char* name;
  uintptr_t st;
  float t0, t1;
};
constexpr size_t kProfSpanCap = 1u << 20;
struct ProfTotal {
  uint64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
  double units = 0.0;
};
static std::mutex g_prof_mu;
static std::vector<ProfPending> g_prof_pending;
static std::vector<cudaEvent_t> g_prof_free;
static std::map<std::string, ProfTotal> g_prof_tot;
static std::vector<ProfSpan> g_prof_spans;
static cudaEvent_t g_prof_base = nullptr;

static cudaEvent_t prof_event() {
  cudaEvent_t e = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_free.empty()) {
      e = g_prof_free.back();
      g_prof_free.pop_back();
      return e;
    }
  }
  cudaEventCreate(&e);
  return e;
}

// Inside stream capture the records become event-record nodes of the graph
// (external records), so launches inside graphs are timed too.
static void prof_record(cudaEvent_t e, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
  else
    cudaEventRecord(e, st);
}

void prof_begin(cudaStream_t st, cudaEvent_t* a) {
  *a = prof_event();
  prof_record(*a, st);
}

void prof_end(const char* name, cudaStream_t st, cudaEvent_t a) {
  cudaEvent_t b = prof_event();
  prof_record(b, st);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_pending.push_back(ProfPending{name, a, b, st});
}

void prof_add_work(const char* name, double bytes, double units) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfTotal& t = g_prof_tot[name];
  t.bytes += bytes;
  t.units += units;
}

// Work whose size is only known on the device (records a kernel emitted): the
// count is copied to a page-locked slot on the stream and read when the
// profile is collected, so no synchronisation is added to the pass.
struct ProfCount {
  const char* name;
  cudaEvent_t e;
  unsigned long long* slot;
  double bytes, per, units, units_per;
};
static std::vector<ProfCount> g_prof_counts;
static std::vector<unsigned long long*> g_prof_slots;   // free page-locked slots

void prof_add_work_async(const char* name, const unsigned long long* d_count, double bytes, double bytes_per_count,
                         double units, double units_per_count, cudaStream_t st) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  unsigned long long* slot = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_slots.empty()) {
      constexpr int kChunk = 256;
      unsigned long long* chunk = nullptr;
      if (cudaHostAlloc((void**)&chunk, kChunk * sizeof(unsigned long long), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
      for (int i = 0; i < kChunk; ++i) g_prof_slots.push_back(chunk + i);
    }
    slot = g_prof_slots.back();
    g_prof_slots.pop_back();
  }
  cudaEvent_t e = prof_event();
  cudaMemcpyAsync(slot, d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
  cudaEventRecord(e, st);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_counts.push_back(ProfCount{name, e, slot, bytes, bytes_per_count, units, units_per_count});
}

static void prof_collect() {
  std::vector<ProfPending> pend;
  std::vector<ProfCount> counts;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    pend.swap(g_prof_pending);
    counts.swap(g_prof_counts);
  }
  for (auto& c : counts) {
    cudaEventSynchronize(c.e);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfTotal& t = g_prof_tot[c.name];
    t.bytes += c.bytes + c.per * (double)*c.slot;
    t.units += c.units + c.units_per * (double)*c.slot;
    g_prof_free.push_back(c.e);
    g_prof_slots.push_back(c.slot);
  }
  for (auto& p : pend) {
    float ms = 0.0f, t0 = 0.0f;
    cudaEventSynchronize(p.b);
    cudaEventElapsedTime(&ms, p.a, p.b);
    const bool span = g_prof_base && cudaEventElapsedTime(&t0, g_prof_base, p.a) == cudaSuccess;
    if (!span) cudaGetLastError();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (span && g_prof_spans.size() < kProfSpanCap)
      g_prof_spans.push_back(ProfSpan{p.name, reinterpret_cast<uintptr_t>(p.st), t0, t0 + ms});
    ProfTotal& t = g_prof_tot[p.name];
    t.launches++;
    t.ms += ms;
    g_prof_free.push_back(p.a);
    g_prof_free.push_back(p.b);
  }
}

void set_error(const std::string& msg) { t_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
  set_error(buf);
  if (e == cudaErrorMemoryAllocation) return GOD_ENOMEM;
  return GOD_ECUDA;
}

int num_sms() {
  static thread_local int dev_cached = -1, sms = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != dev_cached) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    dev_cached = dev;
  }
  return sms;
}

static std::mutex g_pool_mu;
static bool g_pool_ready[64];

int dmalloc(void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  GOD_CK(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_ready[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ULL;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      g_pool_ready[dev] = true;
    }
  }
  const cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    char buf[160];
    snprintf(buf, sizeof buf, "device allocation of %zu bytes failed (%s)", bytes, cudaGetErrorString(e));
    set_error(buf);
    return GOD_ENOMEM;
  }
  return GOD_OK;
}

void dfree(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// ---- CUDA graphs: capture every call, update the cached executable in place
static std::mutex g_graph_mu;
static std::unordered_map<uint64_t, cudaGraphExec_t> g_graph_exec;

int graph_run(uint64_t key, cudaStream_t st, int (*body)(void*), void* ctx) {
  // the legacy default stream cannot be captured
  if (!g_graphs_on.load(std::memory_order_relaxed) || st == nullptr) return body(ctx);
  int dev = 0;
  GOD_CK(cudaGetDevice(&dev));
  // one executable per (shape key, stream): the same executable is never
  // launched into two streams at once
  key ^= ((uint64_t)(uintptr_t)st * 0x9E3779B97F4A7C15ULL) ^ ((uint64_t)dev << 56);
  cudaGraph_t g = nullptr;
  GOD_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const int rc = body(ctx);
  const cudaError_t ec = cudaStreamEndCapture(st, &g);
  if (rc != GOD_OK) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc;
  }
  if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture", __FILE__, __LINE__);
  cudaError_t e = cudaSuccess;
  {
    std::lock_guard<std::mutex> lk(g_graph_mu);
    cudaGraphExec_t& ex = g_graph_exec[key];
    if (ex) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(ex, g, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(ex);
        ex = nullptr;
      }
    }
    if (!ex) e = cudaGraphInstantiate(&ex, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, st);
  }
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "graph instantiate/launch", __FILE__, __LINE__);
  return GOD_OK;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int parse_pattern(const char* s, PatternInfo* out) {
  if (!s) return GOD_EINVAL;
  const size_t L = strlen(s);
  if (L == 0 || L > (size_t)kMaxPattern) return GOD_EINVAL;
  PatternInfo P{};
  P.p = (int)L;
  P.x = 0;
  P.ones_prefix[0] = 0;
  for (size_t i = 0; i < L; ++i) {
    if (s[i] != '0' && s[i] != '1') return GOD_EINVAL;
    if (s[i] == '1') P.off[P.x++] = (int)i;
    P.ones_prefix[i + 1] = P.x;
  }
  if (P.x == 0) return GOD_EINVAL;
  *out = P;
  return GOD_OK;
}

// ---- ownership registry for god_free
enum class Kind { Index, HostArray, DeviceArray, Slice };
struct Owned {
  Kind kind;
  cudaStream_t stream;
  int device;
  void (*release)(void*);   // Slice: called with ctx when the slice is freed
  void* ctx;
};
static std::mutex g_reg_mu;
static std::unordered_map<void*, Owned> g_reg;

static void reg_add(void* p, Kind k, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_reg_mu);
  g_reg[p] = Owned{k, st, dev, nullptr, nullptr};
}

void register_host_array(void* p) {
  if (p) reg_add(p, Kind::HostArray, 0);
}

void register_slice(void* p, void (*release)(void*), void* ctx) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_reg_mu);
  g_reg[p] = Owned{Kind::Slice, 0, 0, release, ctx};
}

// Device address of page-locked host memory (readable and writable by kernels
// over the host link), null for any other pointer.
static void* pinned_host_device_ptr(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// A host-or-device input as a device-readable pointer: device memory and
// page-locked host memory are used in place (kernels read the latter over the
// host link, once, while they compute), other host memory is copied into a
// device buffer.
static int to_device(const void* p, size_t bytes, DBuf<uint8_t>& hold, const void** dp, cudaStream_t st) {
  if (is_device_ptr(p)) {
    *dp = p;
    return GOD_OK;
  }
  if (void* mapped = pinned_host_device_ptr(p)) {
    *dp = mapped;
    return GOD_OK;
  }
  if (bytes == 0) {   // nothing is read through it
    *dp = p;
    return GOD_OK;
  }
  GOD_TRY(hold.alloc(bytes, st));
  GOD_CK(cudaMemcpyAsync(hold.p, p, bytes, cudaMemcpyHostToDevice, st));
  *dp = hold.p;
  return GOD_OK;
}

static void free_index(god_index* idx) {
  if (!idx) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(idx->device);
  // any stream may still use the index: wait for the device once, then hand
  // the arrays back to the stream-ordered pool (no per-array synchronisation)
  cudaDeviceSynchronize();
  void* arrays[6] = {idx->d_keys, idx->d_start, idx->d_leaves, idx->d_ent, idx->d_ht, idx->d_root};
  for (void* a : arrays)
    if (a) cudaFreeAsync(a, 0);
  cudaSetDevice(prev);
  delete idx;
}

}  // namespace god

using namespace god;

extern "C" {

const char* god_strerror(int rc) {
  switch (rc) {
    case GOD_OK: return "ok";
    case GOD_EINVAL: return "invalid argument";
    case GOD_ENOMEM: return "out of memory";
    case GOD_ECUDA: return "CUDA error";
    case GOD_ETIMEOUT: return "device wait timed out";
    case GOD_ERANGE: return "output buffer too small";
    case GOD_EBUSY: return "request not finished";
    default: return "unknown error";
  }
}

const char* god_last_error(void) { return t_last_error.c_str(); }

uint64_t god_launch_count(void) { return g_launches.load(); }

void god_set_graphs(int on) { g_graphs_on.store(on ? 1 : 0); }

// Called with g_prof_mu held.
static void prof_mark_base() {
  if (!g_prof_base && cudaEventCreate(&g_prof_base) != cudaSuccess) {
    cudaGetLastError();
    g_prof_base = nullptr;
    return;
  }
  cudaEventRecord(g_prof_base, 0);
}

void god_prof_enable(int on) {
  if (!on) {
    prof_collect();
  } else {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_prof_base) prof_mark_base();
  }
  g_prof_on.store(on == 2 ? 2 : (on ? 1 : 0));
}

void god_prof_reset(void) {
  prof_collect();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_tot.clear();
  g_prof_spans.clear();
  prof_mark_base();
}

int god_prof_timeline(char* buf, uint64_t cap) {
  prof_collect();
  std::string out = "[";
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::map<uintptr_t, int> ids;
    for (size_t i = 0; i < g_prof_spans.size(); ++i) {
      const ProfSpan& sp = g_prof_spans[i];
      auto it = ids.find(sp.st);
      const int id = it == ids.end() ? (ids[sp.st] = (int)ids.size()) : it->second;
      char item[256];
      snprintf(item, sizeof item, "%s[\"%s\", %d, %.4f, %.4f]", i ? ", " : "", sp.name, id, sp.t0, sp.t1);
      out += item;
    }
  }
  out += "]";
  if (!buf || cap < out.size() + 1) return (int)(out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return 0;
}

int god_prof_report(char* buf, uint64_t cap) {
  prof_collect();
  std::string out = "{";
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    bool first = true;
    for (auto& kv : g_prof_tot) {
      if (!kv.second.launches) continue;   // work recorded for a kernel that was not timed
      char item[320];
      snprintf(item, sizeof item, "%s\"%s\": [%llu, %.6f, %.1f, %.1f]", first ? "" : ", ", kv.first.c_str(),
               (unsigned long long)kv.second.launches, kv.second.ms, kv.second.bytes, kv.second.units);
      out += item;
      first = false;
    }
  }
  out += "}";
  if (!buf || cap < out.size() + 1) return (int)(out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return 0;
}

void god_params_init(god_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->index_kind = GOD_INDEX_HASH;
  p->pa_t = 32;
  p->rmi_leaf_bits = 0;
  p->rmi_eps_max = 64;
  p->rmi_root = GOD_ROOT_MLP;
  p->rmi_train_steps = 64;
  p->rmi_train_samples = 65536;
  p->tune = 0;
}

void god_seed_opts_init(god_seed_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->pa_t = UINT32_MAX;
  o->via = -1;
}

int god_build_index_ex(const uint8_t* ref, uint64_t len, const char* pattern, int k, int w, uint32_t max_occ,
                       const god_params* params, void* stream, god_index** out) {
  if (!out) return GOD_EINVAL;
  *out = nullptr;
  PatternInfo P;
  if (parse_pattern(pattern, &P) != GOD_OK) { set_error("pattern must be 1..64 characters of 0/1 with at least one 1"); return GOD_EINVAL; }
  if (k < 1 || k > 28) { set_error("k must be in [1, 28]"); return GOD_EINVAL; }
  if (w < 1 || w > 255) { set_error("w must be in [1, 255]"); return GOD_EINVAL; }
  if (max_occ < 1) { set_error("max_occ must be >= 1"); return GOD_EINVAL; }
  if (len >= (1ULL << 32)) { set_error("reference must be shorter than 2^32 bases"); return GOD_EINVAL; }
  if (len > 0 && !ref) { set_error("null reference"); return GOD_EINVAL; }
  god_params prm;
  god_params_init(&prm);
  if (params) prm = *params;
  if (prm.rmi_eps_max > 254) prm.rmi_eps_max = 254;
  cudaStream_t st = (cudaStream_t)stream;
  god_index* idx = new god_index();
  memset(idx, 0, sizeof(*idx));
  cudaGetDevice(&idx->device);
  idx->pat = P;
  strncpy(idx->pattern, pattern, kMaxPattern);
  idx->k = k;
  idx->w = w;
  idx->max_occ = max_occ;
  idx->ref_len = len;
  idx->params = prm;
  DBuf<uint8_t> hold;
  const void* dref = nullptr;
  int rc = to_device(ref, len, hold, &dref, st);
  if (rc == GOD_OK) rc = build_index_device(idx, (const uint8_t*)dref, len, st);
  if (rc == GOD_OK && prm.index_kind == GOD_INDEX_LEARNED) rc = build_rmi(idx, st);
  if (rc == GOD_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "build sync", __FILE__, __LINE__);
  }
  if (rc != GOD_OK) {
    free_index(idx);
    return rc;
  }
  reg_add(idx, Kind::Index, st);
  *out = idx;
  return GOD_OK;
}

int god_build_index(const uint8_t* ref, uint64_t len, const char* pattern, int k, int w, uint32_t max_occ,
                    god_index** out) {
  return god_build_index_ex(ref, len, pattern, k, w, max_occ, nullptr, nullptr, out);
}

int god_index_get_info(const god_index* idx, god_index_info* info) {
  if (!idx || !info) return GOD_EINVAL;
  memset(info, 0, sizeof(*info));
  info->ref_len = idx->ref_len;
  info->n_minimizers = idx->n_min;
  info->n_keys = idx->n_keys;
  info->n_entries = idx->n_ent;
  info->ht_capacity = idx->ht_cap;
  info->k = idx->k;
  info->w = idx->w;
  info->p = idx->pat.p;
  info->x = idx->pat.x;
  info->max_occ = idx->max_occ;
  info->has_learned = idx->has_rmi;
  info->rmi_leaves = idx->has_rmi ? idx->root.n_leaves : 0;
  info->rmi_fallback_leaves = idx->rmi_fallback_leaves;
  info->rmi_mean_eps = idx->rmi_mean_eps;
  info->rmi_max_eps = idx->rmi_max_eps;
  info->rmi_fallback_key_frac = idx->rmi_fallback_key_frac;
  info->rmi_final_loss = idx->rmi_loss;
  info->device_bytes = idx->device_bytes;
  return GOD_OK;
}

int god_index_export(const god_index* idx, uint64_t* keys, uint64_t* start, uint64_t* entries) {
  if (!idx) return GOD_EINVAL;
  if (keys && idx->n_keys) GOD_CK(cudaMemcpy(keys, idx->d_keys, idx->n_keys * 8, cudaMemcpyDefault));
  if (start) {
    uint32_t* tmp = (uint32_t*)malloc((idx->n_keys + 1) * 4);
    if (!tmp) return GOD_ENOMEM;
    cudaError_t e = cudaMemcpy(tmp, idx->d_start, (idx->n_keys + 1) * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) { free(tmp); return cuda_fail(e, "export start", __FILE__, __LINE__); }
    for (uint64_t i = 0; i <= idx->n_keys; ++i) start[i] = tmp[i];
    free(tmp);
  }
  if (entries && idx->n_ent) GOD_CK(cudaMemcpy(entries, idx->d_ent, idx->n_ent * 8, cudaMemcpyDefault));
  return GOD_OK;
}

namespace {
__global__ void split_sc(const uint64_t* sc, uint64_t n, uint32_t* count, uint64_t* first) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (count) count[i] = (uint32_t)(sc[i] >> 32);
    if (first) first[i] = (uint32_t)sc[i];
  }
}
__global__ void split_minrec(const MinRec* r, uint64_t n, uint64_t* keys, uint32_t* pos, uint8_t* z) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    if (keys) keys[i] = r[i].key;
    if (pos) pos[i] = r[i].pos;
    if (z) z[i] = (uint8_t)(r[i].segz & 1u);
  }
}
}  // namespace

int god_index_lookup(const god_index* idx, const uint64_t* keys, uint64_t n, int via, uint32_t* count,
                     uint64_t* first, void* stream) {
  if (!idx || (n && !keys)) return GOD_EINVAL;
  if (via == 1 && !idx->has_rmi) { set_error("index has no learned part"); return GOD_EINVAL; }
  if (n == 0) return GOD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  DBuf<uint8_t> hold;
  const void* dk = nullptr;
  GOD_TRY(to_device(keys, n * 8, hold, &dk, st));
  DBuf<uint64_t> sc;
  GOD_TRY(sc.alloc(n, st));
  GOD_TRY(lookup_keys(device_view(idx, via), (const uint64_t*)dk, 8, n, via, sc.p, st));
  const bool dev_out = is_device_ptr(count ? (const void*)count : (const void*)first);
  if (dev_out) {
    GOD_LAUNCH(split_sc, 1024, 256, 0, st, sc.p, n, count, first);
    GOD_CK(cudaStreamSynchronize(st));
    return GOD_OK;
  }
  DBuf<uint32_t> dc;
  DBuf<uint64_t> df;
  GOD_TRY(dc.alloc(n, st));
  GOD_TRY(df.alloc(n, st));
  GOD_LAUNCH(split_sc, 1024, 256, 0, st, sc.p, n, dc.p, df.p);
  if (count) GOD_CK(cudaMemcpyAsync(count, dc.p, n * 4, cudaMemcpyDeviceToHost, st));
  if (first) GOD_CK(cudaMemcpyAsync(first, df.p, n * 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  return GOD_OK;
}

int god_sketch(const uint8_t* seq, uint64_t len, const char* pattern, uint32_t shift, int k, int w, uint64_t* keys,
               uint32_t* pos, uint8_t* z, uint64_t cap, uint64_t* n_out, void* stream) {
  if (!n_out) return GOD_EINVAL;
  *n_out = 0;
  PatternInfo P;
  if (parse_pattern(pattern, &P) != GOD_OK || k < 1 || k > 28 || w < 1 || w > 255) return GOD_EINVAL;
  if (len >= (1ULL << 32) || (len && !seq)) return GOD_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  DBuf<uint8_t> hold;
  const void* ds = nullptr;
  GOD_TRY(to_device(seq, len, hold, &ds, st));
  const uint64_t m = patterned_len(P, len, shift);
  DBuf<SegDesc> seg;
  DBuf<uint64_t> voff;
  GOD_TRY(seg.alloc(1, st));
  GOD_TRY(voff.alloc(2, st));
  SegDesc hs{0, (uint32_t)m, 0, shift, 0};
  uint64_t hv[2] = {0, m + 1};
  GOD_CK(cudaMemcpyAsync(seg.p, &hs, sizeof hs, cudaMemcpyHostToDevice, st));
  GOD_CK(cudaMemcpyAsync(voff.p, hv, sizeof hv, cudaMemcpyHostToDevice, st));
  SketchJob job{};
  job.bytes = (const uint8_t*)ds;
  job.segs = seg.p;
  job.seg_voff = voff.p;
  job.n_seg = 1;
  job.V = m + 1;
  job.k = k;
  job.w = w;
  job.pat = P;
  DBuf<MinRec> rec;
  uint64_t total = 0;
  GOD_TRY(run_sketch(job, st, rec, &total, nullptr));
  *n_out = total;
  if (total > cap) return GOD_ERANGE;
  if (total == 0) return GOD_OK;
  DBuf<uint64_t> dk;
  DBuf<uint32_t> dp;
  DBuf<uint8_t> dz;
  GOD_TRY(dk.alloc(total, st));
  GOD_TRY(dp.alloc(total, st));
  GOD_TRY(dz.alloc(total, st));
  GOD_LAUNCH(split_minrec, 1024, 256, 0, st, rec.p, total, dk.p, dp.p, dz.p);
  if (keys) GOD_CK(cudaMemcpyAsync(keys, dk.p, total * 8, cudaMemcpyDefault, st));
  if (pos) GOD_CK(cudaMemcpyAsync(pos, dp.p, total * 4, cudaMemcpyDefault, st));
  if (z) GOD_CK(cudaMemcpyAsync(z, dz.p, total, cudaMemcpyDefault, st));
  GOD_CK(cudaStreamSynchronize(st));
  return GOD_OK;
}

static int seed_common(const god_index* idx, const uint8_t* reads, const uint64_t* offsets, uint32_t n,
                       const god_seed_opts& o, god_anchor** d_alloc, uint64_t* n_anchors, god_anchor* user_dev,
                       uint64_t user_cap) {
  cudaStream_t st = (cudaStream_t)o.stream;
  if (!idx || !n_anchors || (n && (!reads || !offsets))) return GOD_EINVAL;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != idx->device) { set_error("index belongs to another device"); return GOD_EINVAL; }
  *n_anchors = 0;
  if (n == 0) return GOD_OK;
  DBuf<uint8_t> hold_off, hold_reads;
  const void* doff = nullptr;
  const void* dreads = nullptr;
  uint64_t bytes = 0;
  if (is_device_ptr(offsets)) {
    doff = offsets;
    // the total is needed only to copy reads from pageable host memory
    if (!is_device_ptr(reads) && !pinned_host_device_ptr(reads)) {
      GOD_CK(cudaMemcpyAsync(&bytes, offsets + n, 8, cudaMemcpyDeviceToHost, st));
      GOD_CK(cudaStreamSynchronize(st));
    }
  } else {
    // the offsets themselves are checked on the device (make_pa_segments);
    // only the total is needed here, to size the copy of the reads
    if (offsets[n] < offsets[0]) {
      set_error("offsets must be non-decreasing and each read < 2^31 bytes");
      return GOD_EINVAL;
    }
    bytes = offsets[n];
    GOD_TRY(to_device(offsets, (uint64_t)(n + 1) * 8, hold_off, &doff, st));
  }
  GOD_TRY(to_device(reads, bytes, hold_reads, &dreads, st));
  if (o.seg_len > 0)
    return seed_segmented(idx, (const uint8_t*)dreads, (const uint64_t*)doff, n, bytes, o, st, d_alloc, n_anchors,
                          user_dev, user_cap, true);
  return seed_device(idx, (const uint8_t*)dreads, (const uint64_t*)doff, n, bytes, o, st, d_alloc, n_anchors,
                     user_dev, user_cap, true);
}

int god_seed_device(const god_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint32_t n,
                    god_anchor** d_anchors, uint64_t* n_anchors, const god_seed_opts* opts) {
  if (!d_anchors) return GOD_EINVAL;
  *d_anchors = nullptr;
  god_seed_opts o;
  god_seed_opts_init(&o);
  if (opts) o = *opts;
  god_anchor* out = nullptr;
  int rc = seed_common(idx, d_reads, d_offsets, n, o, &out, n_anchors, nullptr, 0);
  if (rc != GOD_OK) {
    if (out) dfree(out, (cudaStream_t)o.stream);
    return rc;
  }
  if (!out) GOD_TRY(dmalloc((void**)&out, sizeof(god_anchor), (cudaStream_t)o.stream));
  reg_add(out, Kind::DeviceArray, (cudaStream_t)o.stream);
  *d_anchors = out;
  return GOD_OK;
}

int god_seed_into(const god_index* idx, const uint8_t* reads, const uint64_t* offsets, uint32_t n, god_anchor* out,
                  uint64_t cap, uint64_t* n_anchors, const god_seed_opts* opts) {
  god_seed_opts o;
  god_seed_opts_init(&o);
  if (opts) o = *opts;
  cudaStream_t st = (cudaStream_t)o.stream;
  // a host output (page-locked or not) is filled by one copy after the device
  // pass: the fill kernels writing over the host link measured slower
  if (out && is_device_ptr(out)) {
    int rc = seed_common(idx, reads, offsets, n, o, nullptr, n_anchors, out, cap);
    if (rc == GOD_OK) GOD_CK(cudaStreamSynchronize(st));
    return rc;
  }
  god_anchor* dtmp = nullptr;
  int rc = seed_common(idx, reads, offsets, n, o, &dtmp, n_anchors, nullptr, 0);
  if (rc == GOD_OK && *n_anchors > cap) rc = GOD_ERANGE;
  if (rc == GOD_OK && *n_anchors) {
    if (!out) rc = GOD_EINVAL;
    else {
      cudaError_t e = cudaMemcpyAsync(out, dtmp, *n_anchors * sizeof(god_anchor), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = cuda_fail(e, "anchors D2H", __FILE__, __LINE__);
    }
  }
  if (dtmp) dfree(dtmp, st);
  if (rc == GOD_OK) GOD_CK(cudaStreamSynchronize(st));
  return rc;
}

int god_seed(const god_index* idx, const uint8_t* reads, const uint64_t* offsets, uint32_t n, god_anchor** anchors,
             uint64_t* n_anchors) {
  if (!anchors || !n_anchors) return GOD_EINVAL;
  *anchors = nullptr;
  god_seed_opts o;
  god_seed_opts_init(&o);
  god_anchor* dtmp = nullptr;
  int rc = seed_common(idx, reads, offsets, n, o, &dtmp, n_anchors, nullptr, 0);
  if (rc != GOD_OK) {
    if (dtmp) dfree(dtmp, 0);
    return rc;
  }
  god_anchor* h = (god_anchor*)malloc(std::max<uint64_t>(*n_anchors, 1) * sizeof(god_anchor));
  if (!h) {
    if (dtmp) dfree(dtmp, 0);
    return GOD_ENOMEM;
  }
  if (*n_anchors) {
    cudaError_t e = cudaMemcpy(h, dtmp, *n_anchors * sizeof(god_anchor), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      free(h);
      dfree(dtmp, 0);
      return cuda_fail(e, "anchors D2H", __FILE__, __LINE__);
    }
  }
  if (dtmp) dfree(dtmp, 0);
  GOD_CK(cudaStreamSynchronize(0));
  reg_add(h, Kind::HostArray, 0);
  *anchors = h;
  return GOD_OK;
}

int god_vote(const god_anchor* anchors, uint64_t n_anchors, const uint64_t* offsets, uint32_t n_reads,
             const god_vote_params* params, god_vote_rec* out, uint32_t* counts, void* stream) {
  if (!params || (n_reads && (!offsets || !out || !counts)) || (n_anchors && !anchors)) {
    set_error("god_vote: null argument");
    return GOD_EINVAL;
  }
  if (params->V < 1 || params->max_out < 1 || params->max_out > 32) {
    set_error("god_vote: V must be >= 1 and max_out in 1..32");
    return GOD_EINVAL;
  }
  if (n_reads == 0) return GOD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev_out = is_device_ptr(out);
  if (dev_out != is_device_ptr(counts)) {
    set_error("god_vote: out and counts must both be device or both host memory");
    return GOD_EINVAL;
  }
  if ((dev_out && ((reinterpret_cast<uintptr_t>(out) & 7u) || (reinterpret_cast<uintptr_t>(counts) & 3u))) ||
      (is_device_ptr(anchors) && (reinterpret_cast<uintptr_t>(anchors) & 3u)) ||
      (is_device_ptr(offsets) && (reinterpret_cast<uintptr_t>(offsets) & 7u))) {
    set_error("god_vote: misaligned device array");
    return GOD_EINVAL;
  }
  DBuf<uint8_t> hold_a, hold_o;
  const void* da = nullptr;
  const void* doff = nullptr;
  GOD_TRY(to_device(anchors, n_anchors * sizeof(god_anchor), hold_a, &da, st));
  GOD_TRY(to_device(offsets, ((uint64_t)n_reads + 1) * 8, hold_o, &doff, st));
  if (dev_out) {
    GOD_TRY(vote_device((const god_anchor*)da, n_anchors, (const uint64_t*)doff, n_reads, *params, out, counts, st));
    GOD_CK(cudaStreamSynchronize(st));
    return GOD_OK;
  }
  DBuf<god_vote_rec> dv;
  DBuf<uint32_t> dc;
  GOD_TRY(dv.alloc((uint64_t)n_reads * params->max_out, st));
  GOD_TRY(dc.alloc(n_reads, st));
  GOD_TRY(vote_device((const god_anchor*)da, n_anchors, (const uint64_t*)doff, n_reads, *params, dv.p, dc.p, st));
  GOD_CK(cudaMemcpyAsync(counts, dc.p, (uint64_t)n_reads * 4, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaMemcpyAsync(out, dv.p, (uint64_t)n_reads * params->max_out * sizeof(god_vote_rec), cudaMemcpyDeviceToHost,
                         st));
  GOD_CK(cudaStreamSynchronize(st));
  return GOD_OK;
}

void god_contain_params_init(god_contain_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->pattern = "10";
  p->k = 28;
  p->w = 40;
  p->max_occ = 1000;
  p->pa_t = 32;
  p->D = 100;
  p->V = 3;
  p->index_kind = GOD_INDEX_HASH;
  p->batch_bases = (1ull << 32) - 1;
}

int god_contain(const uint8_t* db, const uint64_t* contig_offsets, uint32_t n_contigs, const uint32_t* contig_genome,
                uint32_t n_genomes, const uint8_t* reads, const uint64_t* read_offsets, uint32_t n_reads,
                const god_contain_params* params, int32_t* read_genome, uint32_t* read_votes, uint64_t* genome_reads,
                uint64_t* genome_bases, void* stream) {
  if (!params || !contig_offsets || (n_contigs && !contig_genome) || (n_reads && (!read_offsets || !reads)) ||
      (n_reads && (!read_genome || !read_votes)) || (n_genomes && (!genome_reads || !genome_bases))) {
    set_error("god_contain: null argument");
    return GOD_EINVAL;
  }
  PatternInfo P;
  if (parse_pattern(params->pattern, &P) != GOD_OK || params->k < 1 || params->k > 28 || params->w < 1 ||
      params->w > 255 || params->V < 1 || params->max_occ < 1 || params->batch_bases == 0) {
    set_error("god_contain: bad pattern, k, w, max_occ, V or batch size");
    return GOD_EINVAL;
  }
  if (is_device_ptr(contig_offsets) || is_device_ptr(contig_genome)) {
    set_error("god_contain: contig offsets and genome ids must be host arrays");
    return GOD_EINVAL;
  }
  for (uint32_t j = 0; j < n_contigs; ++j) {
    if (contig_genome[j] >= n_genomes || contig_offsets[j + 1] < contig_offsets[j]) {
      set_error("god_contain: genome id out of range or decreasing contig offsets");
      return GOD_EINVAL;
    }
  }
  if (contig_offsets[n_contigs] > contig_offsets[0] && !db) {
    set_error("god_contain: null database");
    return GOD_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  DBuf<uint8_t> hold_off, hold_reads;
  const void* doff = nullptr;
  const void* dreads = nullptr;
  uint64_t bytes = 0;
  if (n_reads) {
    if (is_device_ptr(read_offsets)) {
      doff = read_offsets;
      GOD_CK(cudaMemcpyAsync(&bytes, read_offsets + n_reads, 8, cudaMemcpyDeviceToHost, st));
      GOD_CK(cudaStreamSynchronize(st));
    } else {
      bytes = read_offsets[n_reads];
      GOD_TRY(to_device(read_offsets, ((uint64_t)n_reads + 1) * 8, hold_off, &doff, st));
    }
    GOD_TRY(to_device(reads, bytes, hold_reads, &dreads, st));
  }
  return contain_device(db, is_device_ptr(db), contig_offsets, n_contigs, contig_genome, n_genomes,
                        (const uint8_t*)dreads, (const uint64_t*)doff, n_reads, bytes, *params, read_genome,
                        read_votes, genome_reads, genome_bases, st);
}

int god_seed_match(const uint8_t* seqs, const uint64_t* offsets, uint32_t n_pairs, const char* pattern,
                   const char* spaced, int k, int w, uint32_t* ed, uint32_t* matched, uint32_t* total, void* stream) {
  PatternInfo P, SP;
  if (parse_pattern(pattern, &P) != GOD_OK || parse_pattern(spaced, &SP) != GOD_OK || k < 1 || k > 28 || w < 1 ||
      w > 255) {
    set_error("god_seed_match: bad pattern, spaced pattern, k or w");
    return GOD_EINVAL;
  }
  if (n_pairs == 0) return GOD_OK;
  if (!seqs || !offsets || !ed || !matched || !total) {
    set_error("god_seed_match: null argument");
    return GOD_EINVAL;
  }
  const bool dev_out = is_device_ptr(ed);
  if (dev_out != is_device_ptr(matched) || dev_out != is_device_ptr(total)) {
    set_error("god_seed_match: outputs must all be device or all host memory");
    return GOD_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const uint64_t n_off = 2 * (uint64_t)n_pairs + 1;
  DBuf<uint8_t> hold_o, hold_s;
  const void* doff = nullptr;
  const void* dseq = nullptr;
  uint64_t bytes = 0;
  if (is_device_ptr(offsets)) {
    doff = offsets;
    GOD_CK(cudaMemcpyAsync(&bytes, offsets + n_off - 1, 8, cudaMemcpyDeviceToHost, st));
    GOD_CK(cudaStreamSynchronize(st));
  } else {
    bytes = offsets[n_off - 1];
    GOD_TRY(to_device(offsets, n_off * 8, hold_o, &doff, st));
  }
  GOD_TRY(to_device(seqs, bytes, hold_s, &dseq, st));
  if (dev_out)
    return seed_match_device((const uint8_t*)dseq, (const uint64_t*)doff, n_pairs, P, SP, k, w, ed, matched, total,
                             st);
  DBuf<uint32_t> de, dm, dt;
  GOD_TRY(de.alloc(n_pairs, st));
  GOD_TRY(dm.alloc(4 * (uint64_t)n_pairs, st));
  GOD_TRY(dt.alloc(4 * (uint64_t)n_pairs, st));
  GOD_TRY(seed_match_device((const uint8_t*)dseq, (const uint64_t*)doff, n_pairs, P, SP, k, w, de.p, dm.p, dt.p, st));
  GOD_CK(cudaMemcpyAsync(ed, de.p, (uint64_t)n_pairs * 4, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaMemcpyAsync(matched, dm.p, (uint64_t)n_pairs * 16, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaMemcpyAsync(total, dt.p, (uint64_t)n_pairs * 16, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  return GOD_OK;
}

int god_rmi_root_grad(const float* theta, int H, const float* x, const float* y, uint64_t n, float* grad, float* loss) {
  if (!theta || !grad || !loss || (n && (!x || !y)) || H != kRootHidden) return GOD_EINVAL;
  const int np = 3 * H + 1;
  DBuf<float> dt, dx, dy, dg, dl;
  GOD_TRY(dt.alloc(np, 0));
  GOD_TRY(dx.alloc(n, 0));
  GOD_TRY(dy.alloc(n, 0));
  GOD_TRY(dg.alloc(np, 0));
  GOD_TRY(dl.alloc(1, 0));
  GOD_CK(cudaMemcpy(dt.p, theta, np * 4, cudaMemcpyHostToDevice));
  if (n) {
    GOD_CK(cudaMemcpy(dx.p, x, n * 4, cudaMemcpyHostToDevice));
    GOD_CK(cudaMemcpy(dy.p, y, n * 4, cudaMemcpyHostToDevice));
  }
  GOD_TRY(rmi_root_grad_device(dt.p, H, dx.p, dy.p, n, dg.p, dl.p, 0));
  GOD_CK(cudaMemcpy(grad, dg.p, np * 4, cudaMemcpyDeviceToHost));
  GOD_CK(cudaMemcpy(loss, dl.p, 4, cudaMemcpyDeviceToHost));
  return GOD_OK;
}

void god_free(void* p) {
  if (!p) return;
  Owned o;
  {
    std::lock_guard<std::mutex> lk(g_reg_mu);
    auto it = g_reg.find(p);
    if (it == g_reg.end()) return;
    o = it->second;
    g_reg.erase(it);
  }
  switch (o.kind) {
    case Kind::Index: free_index(static_cast<god_index*>(p)); break;
    case Kind::HostArray: free(p); break;
    case Kind::Slice: o.release(o.ctx); break;
    case Kind::DeviceArray: {
      int prev = 0;
      cudaGetDevice(&prev);
      cudaSetDevice(o.device);
      cudaFreeAsync(p, o.stream);
      cudaSetDevice(prev);
      break;
    }
  }
}

}  // extern "C"
