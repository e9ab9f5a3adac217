// Internal declarations shared by the CUDA translation units of libgod.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/god.h"

namespace god {

// ------------------------------------------------------------------ errors
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define GOD_CK(call)                                                        \
  do {                                                                      \
    cudaError_t _e = (call);                                                \
    if (_e != cudaSuccess) return ::god::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define GOD_TRY(call)                 \
  do {                                \
    int _rc = (call);                 \
    if (_rc != GOD_OK) return _rc;    \
  } while (0)

extern std::atomic<uint64_t> g_launches;
extern std::atomic<int> g_prof_on;
// Opt-in per-kernel timing: an event pair around each launch, resolved later.
// Mode 1 times every launch, mode 2 only the sketch kernels' ("sketch", the
// tile kernel, and "sketch_seg", the per-segment kernel).
inline bool prof_wants(const char* kernel) {
  const int m = g_prof_on.load(std::memory_order_relaxed);
  if (m == 1) return true;
  if (m != 2) return false;
  const char* s = "sketch";
  while (*s && *kernel == *s) ++s, ++kernel;
  if (*s) return false;
  if (*kernel == 0) return true;
  const char* t = "_seg";
  while (*t && *kernel == *t) ++t, ++kernel;
  return *t == 0 && *kernel == 0;
}
void prof_begin(cudaStream_t st, cudaEvent_t* a);
void prof_end(const char* name, cudaStream_t st, cudaEvent_t a);
// Adds algorithmic bytes (and processed units) to a kernel's profile entry.
void prof_add_work(const char* name, double bytes, double units);
// The same, with bytes + bytes_per_count x n and units + units_per_count x n,
// n = *d_count: a device counter copied on the stream without synchronising
// and resolved when the profile is read.
void prof_add_work_async(const char* name, const unsigned long long* d_count, double bytes, double bytes_per_count,
                         double units, double units_per_count, cudaStream_t st);

// Every kernel launch goes through this macro: it counts the launch, times it
// when profiling is on, and turns a launch failure into GOD_ECUDA.
#define GOD_LAUNCH(kernel, grid, block, smem, stream, ...)                       \
  do {                                                                           \
    cudaEvent_t _pa = nullptr;                                                   \
    if (::god::prof_wants(#kernel)) ::god::prof_begin((stream), &_pa);            \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                  \
    ::god::g_launches.fetch_add(1, std::memory_order_relaxed);                   \
    cudaError_t _le = cudaGetLastError();                                        \
    if (_pa) ::god::prof_end(#kernel, (stream), _pa);                            \
    if (_le != cudaSuccess) return ::god::cuda_fail(_le, #kernel, __FILE__, __LINE__); \
  } while (0)

int num_sms();

// ------------------------------------------------------------------ memory
// Stream-ordered device allocation (cudaMallocAsync on the device's default
// pool, kept cached by a high release threshold).
int dmalloc(void** p, size_t bytes, cudaStream_t st);
void dfree(void* p, cudaStream_t st);

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t st = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  int alloc(size_t count, cudaStream_t s) {
    release();
    st = s;
    n = count;
    if (count == 0) count = 1;
    return dmalloc((void**)&p, count * sizeof(T), s);
  }
  void release() {
    if (p) dfree(p, st);
    p = nullptr;
    n = 0;
  }
  T* take() {
    T* r = p;
    p = nullptr;
    n = 0;
    return r;
  }
};

bool is_device_ptr(const void* p);
// Hands a malloc'ed host array to god_free's ownership registry.
void register_host_array(void* p);
// Hands a pointer into a shared buffer to god_free: freeing it calls release(ctx).
void register_slice(void* p, void (*release)(void*), void* ctx);

// ------------------------------------------------------------------ pattern
constexpr int kMaxPattern = 64;
struct PatternInfo {
  int p;                       // pattern length
  int x;                       // weight (number of 1s)
  int off[kMaxPattern];        // offsets of the 1s, ascending
  int ones_prefix[kMaxPattern + 1];  // ones in P[0:i]
};
int parse_pattern(const char* s, PatternInfo* out);

// Patterned length of a sequence of `len` bases under shift s (Sec. 3.2):
// x * floor((len - s) / p) + ones(P[0 : (len - s) mod p]).
__host__ __device__ inline uint64_t patterned_len(const PatternInfo& P, uint64_t len, uint32_t s) {
  if (len <= s) return 0;
  const uint64_t L = len - s;
  return (uint64_t)P.x * (L / (uint64_t)P.p) + (uint64_t)P.ones_prefix[L % (uint64_t)P.p];
}

// ------------------------------------------------------------------ sketch
// One patterned sequence of the virtual stream processed by the sketch kernel.
struct SegDesc {
  uint64_t byte_off;   // first byte of the source sequence in the byte buffer
  uint32_t m;          // patterned bases of this segment (possibly a prefix)
  uint32_t read;       // owning read (0 for the reference)
  uint32_t shift;      // pattern shift s
  uint32_t flags;      // kSegCapped when m is a prefix of the patterned read
};
constexpr uint32_t kSegCapped = 1u;

// One minimizer: key = H(canonical k-mer); pos = original position of the
// k-mer's first kept base; segz = (segment << 1) | z. 16 bytes.
struct __align__(16) MinRec {
  uint64_t key;
  uint32_t pos;
  uint32_t segz;
};

struct SketchTune {
  int tile;     // owned k-mer positions per warp sub-tile (derived)
  int threads;  // threads per CTA (128 or 256)
  int chunks;   // 8-base chunks per thread per tile (1 or 2)
};

struct SketchJob {
  const uint8_t* bytes;
  const SegDesc* segs;
  const uint64_t* seg_voff;   // n_seg + 1 virtual offsets (each segment m + 1)
  uint32_t n_seg;
  uint64_t V;                 // seg_voff[n_seg], read back by the caller
  int k, w;
  PatternInfo pat;
  MinRec* out;
  uint64_t out_cap;
  uint32_t* seg_cnt;          // optional per-segment minimizer counts (zeroed by caller)
  uint32_t* read_flag;        // optional: set to 1 for reads with an N in a capped segment
  int tune;                   // 1: pick the launch shape with the autotuner (cached per shape class)
  uint32_t max_m;             // longest segment's m when known (0 = unknown); batches of short
                              // segments then run the one-thread-per-segment kernel
  int bytes_on_host;          // 1: `bytes` is page-locked host memory read over the host link
                              // (the per-segment kernel then stages each warp's span with wide loads)
  const uint32_t* own;        // optional (per-segment kernel): segment g emits only the minimizers
                              // whose k-mer index lies in [own[2g], own[2g + 1]) (the reference cut
                              // into overlapping pieces, each owning the k-mers whose windows it holds)
};

// Runs the fused sparsify + 2-bit code + hash + window-minimum kernel over the
// virtual stream and returns its minimizer records in stream order (segment,
// position) in `out`, allocated to exactly *total records. job.out / out_cap
// are not used.
int run_sketch(const SketchJob& job, cudaStream_t st, DBuf<MinRec>& out, uint64_t* total, const SketchTune* tune);

// The same pass without the final compaction: sub-tile s holds sub_cnt[s]
// records at staging[s * WT ...] in stream order; sub_off is their exclusive
// scan (n_sub + 1 entries, sub_off[n_sub] = total). For callers that fuse the
// compaction into their own next pass.
struct StagedSketch {
  DBuf<MinRec> staging;
  DBuf<uint32_t> sub_cnt;
  DBuf<uint64_t> sub_off;
  uint64_t n_sub = 0, total = 0;
  int WT = 0;
  // when set, sub-tile s's records start at staging[sub_base[s]] instead of
  // staging[s * WT] (the per-segment kernel: one sub-tile per segment, based
  // at the segment's virtual offset)
  const uint64_t* sub_base = nullptr;
};
int run_sketch_staged(const SketchJob& job, cudaStream_t st, StagedSketch& out, const SketchTune* tune);
// The one-thread-per-segment kernel (sketch_seg.cu): whether it takes this
// job (seg_cnt set, every segment short, w in {10, 11, 19}), and the pass
// itself: the same records and order as the tile kernel, one sub-tile per
// segment (sub_cnt = the segment counts, sub_off their scan, sub_base =
// seg_voff). The total stays on the device (sub_off[n_sub]); out.total is
// not set.
bool sketch_segments_ok(const SketchJob& job);
int run_sketch_segments(const SketchJob& job, cudaStream_t st, StagedSketch& out);
SketchTune default_sketch_tune(int k, int w);

// ------------------------------------------------------------------ scan
// Exclusive prefix sum of n values into out (n + 1 entries: out[n] = total).
int exclusive_scan_u32(const uint32_t* in, uint64_t* out, uint64_t n, cudaStream_t st);
int exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t st);
// out[n] is ~0 when a look-back wait gave up; callers read it back with their
// next synchronisation and report GOD_ETIMEOUT (scan_total_ok).
constexpr uint64_t kScanPoison = ~0ULL;
inline int scan_total_ok(uint64_t total, const char* what) {
  if (total != kScanPoison) return GOD_OK;
  set_error(std::string(what) + ": prefix-sum wait gave up");
  return GOD_ETIMEOUT;
}
// The same with a caller-provided workspace of scan_ws_words(n) uint64 words
// (no allocation: usable inside stream capture).
uint64_t scan_ws_words(uint64_t n);
int exclusive_scan_u32_ws(const uint32_t* in, uint64_t* out, uint64_t n, uint64_t* ws, cudaStream_t st);

// ------------------------------------------------------------------ graphs
// Runs `body` (a fixed sequence of kernel launches on st, no allocation, no
// host synchronisation) as a CUDA graph: it is captured on every call and the
// executable graph cached under `key` is updated in place (cudaGraphExecUpdate)
// and launched; a topology change re-instantiates it. Direct launches when
// graphs are switched off.
int graph_run(uint64_t key, cudaStream_t st, int (*body)(void*), void* ctx);
extern std::atomic<int> g_graphs_on;

// ------------------------------------------------------------------ radix sort
// Stable LSD radix sort of (key, value) pairs by bits [0, key_bits) of the key.
// keys/vals are sorted in place (alternate buffers are allocated internally).
int radix_sort_pairs(uint64_t* keys, uint64_t* vals, uint64_t n, int key_bits, cudaStream_t st);
// The same with 32-bit values.
int radix_sort_pairs32(uint64_t* keys, uint32_t* vals, uint64_t n, int key_bits, cudaStream_t st);
// ------------------------------------------------------------------ index
constexpr uint64_t kEmptyKey = ~0ULL;

struct RmiLeaf {               // 16 bytes
  uint64_t base_eps;           // base key (low 56 bits) | error bound (high 8 bits)
  float slope;
  float icept;
};

constexpr int kRootHidden = 32;
struct RmiRoot {
  float W1[kRootHidden];
  float b1[kRootHidden];
  float W2[kRootHidden];
  float b2;
  uint64_t kmin, kmax;
  float inv_span;
  uint32_t n_leaves;
  // The trained 1 -> H -> 1 ReLU network as the piecewise-linear function it
  // is: hinge points hx (ascending, +inf past the last) and, on piece i
  // (hx[i - 1] <= x < hx[i]), f(x) = A[i] x + C[i]. Both the build's routing
  // and every lookup evaluate this form (set by rmi_root_pieces).
  float hx[kRootHidden];
  float A[kRootHidden + 1];
  float C[kRootHidden + 1];
};
// Fills R.hx, R.A, R.C from R.W1, R.b1, R.W2, R.b2 (host).
void rmi_root_pieces(RmiRoot& R);

struct DeviceIndex {           // what lookup kernels need, by value
  const uint64_t* keys;        // n_keys ascending
  const uint32_t* start;       // n_keys + 1
  const uint64_t* ent;         // (pos << 1) | z
  // hash table: 2^ht_lc slots of one word [key >> ht_lc | displacement from
  // the home slot (ht_db bits) | field (ht_rb bits)], ~0 when empty. The
  // field is start << ht_cb | count when ht_cb > 0 (payload slots), else the
  // key's rank in keys
  const uint64_t* ht;
  uint32_t ht_lc, ht_db, ht_rb, ht_cb;
  uint64_t n_keys;
  const RmiLeaf* leaves;       // null without a learned index
  const RmiRoot* root;         // device copy
  uint32_t eps_max;
};

}  // namespace god

struct god_index {
  int device;
  god::PatternInfo pat;
  char pattern[god::kMaxPattern + 1];
  int k, w;
  uint32_t max_occ;
  uint64_t ref_len;
  uint64_t n_min;
  uint64_t n_keys, n_ent;
  uint64_t* d_keys;
  uint32_t* d_start;
  uint64_t* d_ent;
  uint64_t* d_ht;
  uint64_t ht_cap;
  uint32_t ht_lc, ht_db, ht_rb, ht_cb;
  god_params params;
  // learned index
  int has_rmi;
  god::RmiRoot root;
  god::RmiRoot* d_root;
  god::RmiLeaf* d_leaves;
  uint32_t rmi_fallback_leaves, rmi_max_eps;
  double rmi_mean_eps, rmi_fallback_key_frac;
  float rmi_loss;
  uint64_t device_bytes;
};

namespace god {
god::DeviceIndex device_view(const god_index* idx, int via);
// Looks up n record keys: out[i] = start | count << 32 (0 when absent).
int lookup_keys(const DeviceIndex& di, const uint64_t* keys, size_t key_stride_bytes, uint64_t n,
                int via, uint64_t* out, cudaStream_t st);
int build_index_device(god_index* idx, const uint8_t* d_ref, uint64_t len, cudaStream_t st);
int build_rmi(god_index* idx, cudaStream_t st);
int rmi_root_grad_device(const float* d_theta, int H, const float* d_x, const float* d_y, uint64_t n,
                         float* d_grad, float* d_loss, cudaStream_t st);
int seed_device(const god_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint32_t n,
                uint64_t read_bytes, const god_seed_opts& o, cudaStream_t st, god_anchor** d_out,
                uint64_t* n_anchors, god_anchor* user_out, uint64_t user_cap, bool user_out_device);
// seed_device with reads longer than o.seg_len seeded in segments (god_seed_opts.seg_len).
int seed_segmented(const god_index* idx, const uint8_t* d_reads, const uint64_t* d_offsets, uint32_t n,
                   uint64_t read_bytes, const god_seed_opts& o, cudaStream_t st, god_anchor** d_out,
                   uint64_t* n_anchors, god_anchor* user_out, uint64_t user_cap, bool user_out_device);
// Containment search (see god_contain); reads and read offsets on the device.
int contain_device(const uint8_t* db, bool db_on_device, const uint64_t* coff, uint32_t n_contigs, const uint32_t* cgen,
                   uint32_t n_genomes, const uint8_t* d_reads, const uint64_t* d_roff, uint32_t n_reads,
                   uint64_t read_bytes, const god_contain_params& prm, int32_t* h_read_genome,
                   uint32_t* h_read_votes, uint64_t* h_genome_reads, uint64_t* h_genome_bases, cudaStream_t st);
// Seed matching evaluation over device arrays (see god_seed_match).
int seed_match_device(const uint8_t* d_seqs, const uint64_t* d_offs, uint32_t n, const PatternInfo& P,
                      const PatternInfo& SP, int k, int w, uint32_t* d_ed, uint32_t* d_matched, uint32_t* d_total,
                      cudaStream_t st);
// Location voting over device arrays (see god_vote).
int vote_device(const god_anchor* d_a, uint64_t m, const uint64_t* d_offs, uint32_t n, const god_vote_params& p,
                god_vote_rec* d_out, uint32_t* d_counts, cudaStream_t st);
}  // namespace god
