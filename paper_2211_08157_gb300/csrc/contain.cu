// Containment search (Sec. 2.3): a read set is mapped against a database of
// genomes without a pre-built index. The database is indexed on the fly in
// batches of at most batch_bases bases; every batch is indexed, every read is
// seeded against it and location voting picks its best location; over all
// batches a read keeps the location with the most votes (the earlier batch on
// ties), and each genome counts the reads and read bases mapped to it.
//
// A batch lays its contigs end to end, each starting at a multiple of the
// pattern length after at least one N, so that every contig is sparsified
// from its own start and no k-mer or window spans two contigs. A mapping
// location is a voting winner (votes >= V); its genome is that of the contig
// holding the winner's first reference position.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace god {
namespace {

constexpr int kCT = 256;

inline unsigned grid_for(uint64_t n, int per, unsigned cap_mult) {
  uint64_t b = (n + per - 1) / per;
  b = std::max<uint64_t>(b, 1);
  return (unsigned)std::min<uint64_t>(b, (uint64_t)num_sms() * cap_mult);
}

// Copies contig j of the batch (raw bytes [roff[j], roff[j + 1])) to its start
// base[j] in the layout (which is pre-filled with N).
__global__ void contain_layout(const uint8_t* __restrict__ raw, const uint64_t* __restrict__ roff,
                               const uint64_t* __restrict__ base, uint32_t nc, uint8_t* __restrict__ layout) {
  for (uint32_t j = blockIdx.x; j < nc; j += gridDim.x) {
    const uint64_t a = roff[j], len = roff[j + 1] - a, b = base[j];
    for (uint64_t q = threadIdx.x; q < len; q += blockDim.x) layout[b + q] = raw[a + q];
  }
}

// A read's first voting record, when it is a winner with more votes than its
// best so far, becomes its location; its genome is that of the last contig
// starting at or before the winner's first reference position.
__global__ void contain_update(const god_vote_rec* __restrict__ rec, const uint32_t* __restrict__ cnt, uint32_t n,
                               const uint64_t* __restrict__ base, const uint32_t* __restrict__ cgen, uint32_t nc,
                               uint32_t* __restrict__ best_votes, int32_t* __restrict__ best_genome) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    if (cnt[r] == 0) continue;
    const god_vote_rec v = rec[r];
    if (v.rescue || v.votes <= best_votes[r]) continue;
    uint32_t lo = 0, hi = nc;   // last j with base[j] <= ref_lo
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (base[mid] <= v.ref_lo) lo = mid;
      else hi = mid;
    }
    best_votes[r] = v.votes;
    best_genome[r] = (int32_t)cgen[lo];
  }
}

__global__ void contain_tally(const int32_t* __restrict__ best_genome, const uint64_t* __restrict__ roff, uint32_t n,
                              unsigned long long* __restrict__ greads, unsigned long long* __restrict__ gbases) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const int32_t g = best_genome[r];
    if (g < 0) continue;
    atomicAdd(greads + g, 1ull);
    atomicAdd(gbases + g, (unsigned long long)(roff[r + 1] - roff[r]));
  }
}

__global__ void fill_i32(int32_t* p, uint64_t n, int32_t v) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace

int contain_device(const uint8_t* db, bool db_on_device, const uint64_t* coff, uint32_t n_contigs, const uint32_t* cgen,
                   uint32_t n_genomes, const uint8_t* d_reads, const uint64_t* d_roff, uint32_t n_reads,
                   uint64_t read_bytes, const god_contain_params& prm, int32_t* h_read_genome,
                   uint32_t* h_read_votes, uint64_t* h_genome_reads, uint64_t* h_genome_bases, cudaStream_t st) {
  PatternInfo P;
  GOD_TRY(parse_pattern(prm.pattern, &P));
  const uint64_t p = (uint64_t)P.p;
  DBuf<uint32_t> best_votes;
  DBuf<int32_t> best_genome;
  GOD_TRY(best_votes.alloc(n_reads, st));
  GOD_TRY(best_genome.alloc(n_reads, st));
  if (n_reads) {
    GOD_CK(cudaMemsetAsync(best_votes.p, 0, (size_t)n_reads * 4, st));
    GOD_LAUNCH(fill_i32, grid_for(n_reads, kCT, 16), kCT, 0, st, best_genome.p, n_reads, -1);
  }
  god_params ip;
  god_params_init(&ip);
  ip.index_kind = prm.index_kind;
  ip.pa_t = prm.pa_t;
  god_seed_opts so;
  god_seed_opts_init(&so);
  so.stream = st;
  so.pa_t = prm.pa_t;
  const god_vote_params vp{prm.D, prm.V, 1};
  DBuf<god_vote_rec> vrec;
  DBuf<uint32_t> vcnt;
  GOD_TRY(vrec.alloc(n_reads, st));
  GOD_TRY(vcnt.alloc(n_reads, st));
  uint32_t j0 = 0;
  while (j0 < n_contigs && n_reads) {
    // the batch: contigs [j0, j1) at their starts
    std::vector<uint64_t> base, craw;
    uint64_t end = 0;
    uint32_t j1 = j0;
    while (j1 < n_contigs) {
      const uint64_t b = base.empty() ? 0 : ((end + 1 + p - 1) / p) * p;
      const uint64_t e = b + (coff[j1 + 1] - coff[j1]);
      if (!base.empty() && e > prm.batch_bases) break;
      base.push_back(b);
      craw.push_back(coff[j1] - coff[j0]);
      end = e;
      ++j1;
    }
    craw.push_back(coff[j1] - coff[j0]);
    if (end >= (1ull << 32)) {
      set_error("contain: a contig of 2^32 bases or more");
      return GOD_EINVAL;
    }
    const uint32_t nc = j1 - j0;
    const uint64_t raw_bytes = coff[j1] - coff[j0];
    DBuf<uint8_t> raw, layout;
    DBuf<uint64_t> d_base, d_craw;
    DBuf<uint32_t> d_gen;
    const uint8_t* d_raw = db + coff[j0];
    if (!db_on_device) {
      GOD_TRY(raw.alloc(raw_bytes, st));
      if (raw_bytes) GOD_CK(cudaMemcpyAsync(raw.p, db + coff[j0], raw_bytes, cudaMemcpyHostToDevice, st));
      d_raw = raw.p;
    }
    GOD_TRY(layout.alloc(end, st));
    GOD_TRY(d_base.alloc(nc, st));
    GOD_TRY(d_craw.alloc(nc + 1, st));
    GOD_TRY(d_gen.alloc(nc, st));
    GOD_CK(cudaMemsetAsync(layout.p, 'N', end, st));
    GOD_CK(cudaMemcpyAsync(d_base.p, base.data(), nc * 8, cudaMemcpyHostToDevice, st));
    GOD_CK(cudaMemcpyAsync(d_craw.p, craw.data(), (nc + 1) * 8, cudaMemcpyHostToDevice, st));
    GOD_CK(cudaMemcpyAsync(d_gen.p, cgen + j0, nc * 4, cudaMemcpyHostToDevice, st));
    GOD_LAUNCH(contain_layout, (unsigned)std::min<uint64_t>(nc, (uint64_t)num_sms() * 8), kCT, 0, st, d_raw, d_craw.p,
               d_base.p, nc, layout.p);
    god_index* idx = nullptr;
    int rc = god_build_index_ex(layout.p, end, prm.pattern, prm.k, prm.w, prm.max_occ, &ip, st, &idx);
    if (rc != GOD_OK) return rc;
    god_anchor* anchors = nullptr;
    uint64_t m = 0;
    rc = seed_device(idx, d_reads, d_roff, n_reads, read_bytes, so, st, &anchors, &m, nullptr, 0, true);
    if (rc == GOD_OK) rc = vote_device(anchors, m, d_roff, n_reads, vp, vrec.p, vcnt.p, st);
    if (rc == GOD_OK) {
      contain_update<<<grid_for(n_reads, kCT, 16), kCT, 0, st>>>(vrec.p, vcnt.p, n_reads, d_base.p, d_gen.p, nc,
                                                                  best_votes.p, best_genome.p);
      g_launches.fetch_add(1, std::memory_order_relaxed);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "contain_update", __FILE__, __LINE__);
    }
    if (anchors) dfree(anchors, st);
    if (rc == GOD_OK) {
      const cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = cuda_fail(e, "contain batch", __FILE__, __LINE__);
    }
    god_free(idx);
    if (rc != GOD_OK) return rc;
    j0 = j1;
  }
  DBuf<unsigned long long> tally;
  GOD_TRY(tally.alloc(2 * (uint64_t)n_genomes, st));
  GOD_CK(cudaMemsetAsync(tally.p, 0, 2 * (size_t)n_genomes * 8, st));
  if (n_reads)
    GOD_LAUNCH(contain_tally, grid_for(n_reads, kCT, 16), kCT, 0, st, best_genome.p, d_roff, n_reads, tally.p,
               tally.p + n_genomes);
  if (n_reads) {
    GOD_CK(cudaMemcpyAsync(h_read_genome, best_genome.p, (size_t)n_reads * 4, cudaMemcpyDeviceToHost, st));
    GOD_CK(cudaMemcpyAsync(h_read_votes, best_votes.p, (size_t)n_reads * 4, cudaMemcpyDeviceToHost, st));
  }
  GOD_CK(cudaMemcpyAsync(h_genome_reads, tally.p, (size_t)n_genomes * 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaMemcpyAsync(h_genome_bases, tally.p + n_genomes, (size_t)n_genomes * 8, cudaMemcpyDeviceToHost, st));
  GOD_CK(cudaStreamSynchronize(st));
  return GOD_OK;
}

}  // namespace god
