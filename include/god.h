/*
 * god.h - C ABI of the GB300 Genome-on-Diet seeding library (libgod.so).
 *
 * The library runs the data-parallel hot path of sparsified read mapping
 * (Alser, Eudine & Mutlu, "Genome-on-Diet", arXiv 2211.08157) on one GPU:
 *   - sparsify a sequence with a repeating 0/1 diet pattern (Sec. 3, Sec. 3.1
 *     steps 1-2; shifted patterns in Sec. 3.2),
 *   - 2-bit code the kept bases, N breaking k-mers (Sec. 3.6.1),
 *   - double-strand (w,k)-minimizers with Thomas Wang's integer hash of the
 *     canonical k-mer (Sec. 3.1, Sec. 3.6.1),
 *   - a compressed seed index of the patterned reference with a
 *     high-occurrence filter (Sec. 3.1 step 3, Sec. 3.2),
 *   - pattern alignment of every read (Sec. 3.2) and compressed seeding that
 *     turns the read's minimizers into anchors (Sec. 3.3),
 *   - the anchors of each read sorted, as the voting step expects (Sec. 3.4
 *     step 2).
 * A learned index (a root MLP over the key plus linear leaves with per-leaf
 * error bounds) can replace the hash table for lookup; it returns exactly the
 * hash table's answers.
 *
 * Conventions for every entry point:
 *   - Return value: GOD_OK (0) or a negative GOD_E* code. Nothing aborts or
 *     traps; god_last_error() gives a message for the calling thread.
 *   - Pointers: "host or device" inputs are classified with
 *     cudaPointerGetAttributes; host inputs are copied to the device inside the
 *     call. Inputs are borrowed and never retained after the call returns.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream). Calls that return host results synchronise `stream`.
 *   - Threads: an index is read-only after it is built; concurrent god_seed*
 *     calls on one index are safe when each uses its own stream.
 *   - Device: every call works on the CUDA device that is current on the
 *     calling thread; an index must be used on the device it was built on.
 */
#ifndef GOD_H
#define GOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------- errors */
#define GOD_OK 0
#define GOD_EINVAL -1   /* bad argument: pattern, k, w, sizes, offsets */
#define GOD_ENOMEM -2   /* device or host allocation failed, or admission refused */
#define GOD_ECUDA -3    /* a CUDA runtime error; god_last_error() has its text */
#define GOD_ETIMEOUT -4 /* a bounded device-side wait gave up */
#define GOD_ERANGE -5   /* caller buffer too small; the needed size is returned */
#define GOD_EBUSY -6    /* serving: request not finished yet */

const char *god_strerror(int rc);
/* Message of the last failing call on this thread ("" if none). */
const char *god_last_error(void);

/* ----------------------------------------------------------------- types */
typedef struct god_index god_index; /* opaque; owns its device memory */

/* One anchor: a read minimizer matched to one index entry (Sec. 3.3).
 * read_pos / ref_pos are original (unpatterned) 0-based positions of the
 * first kept base of the k-mer; strand = z_read xor z_ref, where z = 1 when the
 * reverse-complement k-mer is the canonical one. 16 bytes, 4 x u32 little
 * endian. Lists are sorted by (read_id, ref_pos, read_pos, strand). */
typedef struct {
  uint32_t read_id, read_pos, ref_pos, strand;
} god_anchor;

#define GOD_INDEX_HASH 0    /* open-addressing hash table (default) */
#define GOD_INDEX_LEARNED 1 /* learned index, hash table as fallback */

#define GOD_ROOT_MLP 0      /* root = 1 -> 32 -> 1 ReLU MLP trained on the GPU */
#define GOD_ROOT_UNTRAINED 1 /* the same MLP at its initialisation, not trained (ablation) */
#define GOD_ROOT_LINEAR 2    /* no network: leaf = floor(x * leaves), x = normalised key (ablation) */

typedef struct {
  int index_kind;          /* GOD_INDEX_HASH or GOD_INDEX_LEARNED */
  uint32_t pa_t;           /* pattern alignment: first t minimizers per shift (Sec. 3.2); 0 = all. Default 32 */
  int rmi_leaf_bits;       /* learned index: 2^bits leaves, 16..20; 0 = chosen from the key count */
  uint32_t rmi_eps_max;    /* leaves whose error bound exceeds this use the hash table; <= 255. Default 64 */
  int rmi_root;            /* GOD_ROOT_MLP, GOD_ROOT_UNTRAINED or GOD_ROOT_LINEAR */
  int rmi_train_steps;     /* Adam fine-tuning steps after the least-squares readout (0 = the readout
                              alone); default 64 */
  uint32_t rmi_train_samples; /* keys sampled for root training; default 65536 */
  int tune;                /* 1 = autotune the sketch launch (cached per shape); 0 = fixed default */
} god_params;

/* Fills `p` with the defaults above. */
void god_params_init(god_params *p);

/* ----------------------------------------------------------------- index
 * god_build_index: compressed indexing (Sec. 3.1): sparsify `ref` (len bytes,
 * ASCII; any byte outside ACGTacgt is N) with `pattern` at shift 0, compute its
 * (w,k)-minimizers, sort them by (key, position), and keep every key seen at
 * most `max_occ` times (Sec. 3.2 filter). Builds the hash table, and the learned
 * index when params->index_kind says so.
 *   ref      host or device, len bytes; len < 2^32.
 *   pattern  NUL-terminated string of '0'/'1', 1..64 characters, at least one '1'.
 *   k        1..28;  w  1..255;  max_occ >= 1.
 *   out      receives the index; release it with god_free.
 * Errors: GOD_EINVAL for bad arguments, GOD_ENOMEM, GOD_ECUDA, GOD_ETIMEOUT.
 */
int god_build_index(const uint8_t *ref, uint64_t len, const char *pattern, int k, int w,
                    uint32_t max_occ, god_index **out);
int god_build_index_ex(const uint8_t *ref, uint64_t len, const char *pattern, int k, int w,
                       uint32_t max_occ, const god_params *params, void *stream, god_index **out);

typedef struct {
  uint64_t ref_len;
  uint64_t n_minimizers;   /* reference minimizers before the filter */
  uint64_t n_keys;         /* distinct keys kept */
  uint64_t n_entries;      /* (position, strand) entries of kept keys */
  uint64_t ht_capacity;    /* hash-table slots (power of two) */
  int k, w, p, x;          /* seed length, window, pattern length, pattern weight */
  uint32_t max_occ;
  int has_learned;         /* 1 when the learned index was built */
  uint32_t rmi_leaves;     /* number of leaves */
  uint32_t rmi_fallback_leaves; /* leaves routed to the hash table (error bound too large or empty) */
  double rmi_mean_eps;     /* mean error bound over keys (key-weighted) */
  uint32_t rmi_max_eps;    /* largest bound among leaves that do not fall back */
  double rmi_fallback_key_frac; /* share of keys whose leaf falls back */
  float rmi_final_loss;    /* root training loss (MSE on normalised rank) */
  uint64_t device_bytes;   /* device memory held by the index */
} god_index_info;

int god_index_get_info(const god_index *idx, god_index_info *info);

/* Copies the filtered index to host buffers (any may be NULL):
 * keys[n_keys] ascending; start[n_keys + 1] offsets into entries;
 * entries[n_entries] = (ref_pos << 1) | z, ascending within a key. */
int god_index_export(const god_index *idx, uint64_t *keys, uint64_t *start, uint64_t *entries);

/* Exact lookup of n keys (host or device) through the hash table (via = 0) or
 * the learned index (via = 1). count[i] = index entries of keys[i] (0 when
 * absent or filtered), first[i] = offset of the first entry. Output buffers
 * are host or device, like the input. */
int god_index_lookup(const god_index *idx, const uint64_t *keys, uint64_t n, int via,
                     uint32_t *count, uint64_t *first, void *stream);

/* ----------------------------------------------------------------- seeding
 * god_seed: pattern alignment (Sec. 3.2) and compressed seeding (Sec. 3.3) of
 * n reads against `idx`, all reads in one batched pass.
 *   reads    host or device, the reads' bytes back to back.
 *   offsets  host or device, n + 1 uint64 byte offsets (CSR; non-decreasing,
 *            offsets[n] <= bytes in `reads`, each read < 2^31 bytes).
 *   anchors  receives a malloc'ed host array of *n_anchors anchors, sorted by
 *            (read_id, ref_pos, read_pos, strand); release with god_free.
 * For each read and each shift s < p the first t minimizers of the read
 * sparsified at s are looked up; their index counts are summed, and the shift
 * with the largest sum (the smallest such shift on ties, 0 if all are 0) is the
 * read's alignment index a. Every minimizer of the read sparsified at a whose
 * key is kept in the index gives one anchor per index entry.
 */
int god_seed(const god_index *idx, const uint8_t *reads, const uint64_t *offsets, uint32_t n,
             god_anchor **anchors, uint64_t *n_anchors);

typedef struct {
  void *stream;            /* cudaStream_t; NULL = legacy default stream */
  uint32_t pa_t;           /* overrides the index's t when != UINT32_MAX */
  int via;                 /* -1 = the index's kind, 0 = hash, 1 = learned */
  uint32_t *shifts_out;    /* optional host/device array of alignment indices: one per read, or one per
                              segment when seg_len > 0 (read order, then segment order) */
  uint32_t seg_len;        /* 0 = off (default). Otherwise a read longer than seg_len bases is cut into
                              ceil(len / seg_len) consecutive segments of seg_len bases (the last one
                              shorter), as the paper splits ultra-long reads into segments of at most
                              30,000 bases (Sec. 2.2.2); each segment is pattern-aligned on its own
                              (Sec. 3.2) and seeded; its anchors keep the read's id and whole-read
                              positions, and each read's list stays sorted as above */
} god_seed_opts;

void god_seed_opts_init(god_seed_opts *o);

/* As god_seed, writing into a caller buffer `out` (host or device) of `cap`
 * anchors. When cap is too small nothing is written, *n_anchors gets the
 * needed count and GOD_ERANGE is returned. Device outputs are complete when
 * the call returns (the stream is synchronised). */
int god_seed_into(const god_index *idx, const uint8_t *reads, const uint64_t *offsets, uint32_t n,
                  god_anchor *out, uint64_t cap, uint64_t *n_anchors, const god_seed_opts *opts);

/* Device-resident variant: inputs on the device, the anchor array allocated on
 * the device (stream-ordered on opts->stream); release with god_free. */
int god_seed_device(const god_index *idx, const uint8_t *d_reads, const uint64_t *d_offsets,
                    uint32_t n, god_anchor **d_anchors, uint64_t *n_anchors, const god_seed_opts *opts);

/* ----------------------------------------------------------------- sketch
 * Minimizers of one sequence sparsified with (pattern, shift) (Sec. 3.1,
 * Sec. 3.6.1), in ascending patterned position: key, original position of the
 * k-mer's first kept base, strand bit z. `seq` host or device; outputs host or
 * device buffers of `cap` entries (any may be NULL). *n_out = the count; when
 * cap is too small GOD_ERANGE is returned and nothing is written. */
int god_sketch(const uint8_t *seq, uint64_t len, const char *pattern, uint32_t shift, int k, int w,
               uint64_t *keys, uint32_t *pos, uint8_t *z, uint64_t cap, uint64_t *n_out, void *stream);

/* ----------------------------------------------------------------- allocation-free sketch
 * The paper has no counterpart to this entry point; it exists for callers that
 * may not allocate device memory during a call (a host framework whose own
 * allocator owns the device, a latency-critical loop that cannot afford the
 * implicit synchronisation of cudaMalloc/cudaFree, a deployment that forbids
 * allocation after start-up). It returns the same minimizers as god_sketch
 * but calls no cudaMalloc, cudaFree or allocating library routine: the sketch
 * kernel's scratch (ordered-compaction status words, tile ticket, counters,
 * segment descriptor) lives in one 2 MiB device array that every GPU loading
 * the library holds until the process exits.
 *   d_seq    device memory, len bytes (host pointers are rejected: copying
 *            them would need a device buffer).
 *   d_out    device memory for cap records {key, pos, z} (16 bytes each), in
 *            ascending patterned position; the address must be a multiple of
 *            16 bytes (records are written as 16-byte stores), otherwise
 *            GOD_EINVAL is returned before any work.
 *   *n_out   the number of minimizers; when it exceeds cap, only the first cap
 *            records are written and GOD_ERANGE is returned.
 * Sequences whose patterned length (under pattern and shift) exceeds
 * GOD_NOALLOC_MAX_PATTERNED are rejected with GOD_EINVAL before any work.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current and caches it. All calls on
 * a device share the array and each call clears what it needs at its start,
 * so calls that overlap on the GPU (e.g. on two streams) race: serialise
 * them. Every call reads its count back and synchronises its stream before it
 * returns, so it must not be called while that stream is being captured.
 * On GOD_ETIMEOUT (a bounded device wait gave up) *n_out stays 0. */
typedef struct {
  uint64_t key;
  uint32_t pos;
  uint32_t z;
} god_minimizer;

#define GOD_NOALLOC_MAX_PATTERNED 45395007ULL

int god_sketch_noalloc(const uint8_t *d_seq, uint64_t len, const char *pattern, uint32_t shift, int k,
                       int w, god_minimizer *d_out, uint64_t cap, uint64_t *n_out, void *stream);

/* ----------------------------------------------------------------- location voting
 * god_vote: location voting on each read's anchors (Sec. 3.4 steps 1-5,
 * Fig. 8) with the rescue location (Sec. 3.6.3).
 *   1. every anchor is one vote at a signed location v = ref_pos - read_pos
 *      (strand 0) or v = ref_pos - (len - 1 - read_pos) (strand 1: the read
 *      position counted from the read's other end; for an error-free reverse
 *      read this is its reference start minus (k-mer span - 1));
 *   2. the votes of a read are ordered by (strand, v);
 *   3. a group starts at the first vote left and takes every vote of the same
 *      strand with v - v0 <= D; the next group starts at the first vote beyond;
 *   4/5. groups with at least V votes are the read's winners, most votes first
 *      (equal votes in (strand, v0) order), at most max_out of them. Each
 *      record holds the location v0 and its votes (short reads, step 4) and
 *      the reference and read stretches its anchors cover, [ref_lo, ref_hi]
 *      and [read_lo, read_hi] (long reads, step 5);
 *   rescue: when no group reaches V, the group with the most votes (the first
 *      on ties) is reported alone with rescue = 1; a read without anchors
 *      reports nothing.
 *   anchors  host or device, n_anchors records grouped by ascending read_id
 *            (any order inside a read), e.g. a god_seed result; 4-byte aligned.
 *   offsets  host or device, n_reads + 1 CSR byte offsets of the reads (the
 *            read lengths), as given to god_seed.
 *   out      host or device, n_reads * max_out records: read r's are
 *            out[r * max_out + j], j < counts[r]; 8-byte aligned.
 *   counts   host or device (the same kind as out), n_reads entries.
 * Errors: GOD_EINVAL for NULL arrays, V < 1, max_out outside 1..32, a
 * misaligned device array, anchors not grouped by ascending read id or naming
 * a read >= n_reads (found on the device before any result is written), or a
 * read with 2^28 anchors or more; GOD_ENOMEM, GOD_ECUDA. The stream is
 * synchronised before the call returns. */
typedef struct {
  uint32_t read_id, votes, strand, rescue;
  int64_t loc;                          /* v0 */
  uint32_t ref_lo, ref_hi, read_lo, read_hi;
} god_vote_rec;                             /* 40 bytes */

typedef struct {
  uint32_t D;          /* maximum distance from a group's first location */
  uint32_t V;          /* votes a winner needs (>= 1) */
  uint32_t max_out;    /* winners kept per read, 1..32 */
} god_vote_params;

int god_vote(const god_anchor *anchors, uint64_t n_anchors, const uint64_t *offsets, uint32_t n_reads,
             const god_vote_params *params, god_vote_rec *out, uint32_t *counts, void *stream);

/* ----------------------------------------------------------------- containment search
 * god_contain: containment search (Sec. 2.3) of a read set against a database
 * of genomes, without a pre-built index: the database is indexed on the fly in
 * batches of at most batch_bases bases; every read is seeded against each
 * batch (pattern alignment, compressed seeding) and location voting (with D,
 * V) gives its best location there; over all batches a read keeps the winner
 * with the most votes (the earlier batch on ties; a rescue location is not a
 * mapping location here), and each genome counts the reads and read bases
 * mapped to it. A genome's coverage is its mapped read bases / its contig
 * bases; the paper reports genomes with enough mapped reads and coverage >= 1.
 * A batch lays its contigs end to end, each starting at a multiple of the
 * pattern length after at least one N, so every contig is sparsified from its
 * own start and no k-mer spans two contigs; contigs join a batch in database
 * order while its length stays <= batch_bases (at least one per batch; each
 * batch < 2^32 bases).
 *   db              host or device, the contigs' bases back to back.
 *   contig_offsets  host, n_contigs + 1 byte offsets into db.
 *   contig_genome   host, n_contigs genome ids < n_genomes.
 *   reads, read_offsets  host or device, as for god_seed.
 *   read_genome     host, n_reads: genome of each read's location, -1 = unmapped.
 *   read_votes      host, n_reads: votes of that location (0 = unmapped).
 *   genome_reads, genome_bases  host, n_genomes: mapped reads and read bases.
 * Errors: GOD_EINVAL (bad pattern, k, w, V, a genome id out of range,
 * decreasing offsets), GOD_ENOMEM, GOD_ECUDA, GOD_ETIMEOUT. Synchronous. */
typedef struct {
  const char *pattern;     /* default "10" (the paper's containment runs) */
  int k, w;                /* default 28, 40 */
  uint32_t max_occ;        /* default 1000 */
  uint32_t pa_t;           /* pattern alignment minimizers per shift, default 32 */
  uint32_t D, V;           /* location voting, default 100, 3 */
  int index_kind;          /* GOD_INDEX_HASH (default) or GOD_INDEX_LEARNED */
  uint64_t batch_bases;    /* default 2^32 - 1 */
} god_contain_params;

void god_contain_params_init(god_contain_params *p);
int god_contain(const uint8_t *db, const uint64_t *contig_offsets, uint32_t n_contigs,
                const uint32_t *contig_genome, uint32_t n_genomes, const uint8_t *reads,
                const uint64_t *read_offsets, uint32_t n_reads, const god_contain_params *params,
                int32_t *read_genome, uint32_t *read_votes, uint64_t *genome_reads, uint64_t *genome_bases,
                void *stream);

/* ----------------------------------------------------------------- seed matching evaluation
 * god_seed_match: the evaluation of Sec. 2.1.1 / Fig. 4 on n_pairs sequence
 * pairs (S, S') = (sequence 2i, sequence 2i + 1) of at most 1024 bases each:
 *   ed[i]            Levenshtein distance (unit costs, raw bytes);
 *   matched[4i + a]  seeds extracted from S' that occur among S's seeds;
 *   total[4i + a]    seeds extracted from S' (counted with repetition);
 * for a = 0 All Seeds (every k-mer of A/C/G/T bases, forward code),
 * 1 Minimizers ((w,k)-minimizer keys of the unsparsified sequence),
 * 2 Spaced (at every start, the bases under the 1s of `spaced` repeated or
 * cut to k positions), 3 Genome-on-Diet (every k-mer of the sequence
 * sparsified by `pattern` at shift 0). The seed matching rate is
 * matched / total.
 *   seqs, offsets  host or device; offsets has 2 n_pairs + 1 entries.
 *   ed, matched, total  host or device (all the same kind).
 * Errors: GOD_EINVAL (bad patterns, k outside 1..28, w outside 1..255, a
 * sequence longer than 1024 bases or decreasing offsets), GOD_ENOMEM,
 * GOD_ECUDA. Synchronous. */
int god_seed_match(const uint8_t *seqs, const uint64_t *offsets, uint32_t n_pairs, const char *pattern,
                   const char *spaced, int k, int w, uint32_t *ed, uint32_t *matched, uint32_t *total,
                   void *stream);

/* ----------------------------------------------------------------- learned index
 * Gradient of the root MLP's mean squared error (1 -> H -> 1, ReLU; parameter
 * layout W1[H], b1[H], W2[H], b2) over samples (x[i], y[i]), computed by the
 * GPU training kernels. All arrays are host. Returns the loss in *loss. */
int god_rmi_root_grad(const float *theta, int H, const float *x, const float *y, uint64_t n,
                      float *grad, float *loss);

/* ----------------------------------------------------------------- memory
 * Releases an index, or an anchor array returned by god_seed / god_seed_device.
 * NULL is ignored. Anchor arrays are freed stream-ordered on the stream they
 * were allocated on; an index may be in use on any stream, so its release
 * waits for the device once and then returns its arrays to the stream-ordered
 * pool. */
void god_free(void *p);

/* Kernels launched by this library in this process so far. */
uint64_t god_launch_count(void);

/* Opt-in kernel timing: while enabled (on = 1), every launch is bracketed by a
 * pair of CUDA events on its stream; on = 2 times only the sketch kernels'
 * launches ("sketch": the tile kernel; "sketch_seg": one thread per segment) (two events per launch, so the rest of a timed step runs as
 * without timing); 0 switches timing off. god_prof_report writes a JSON object
 * {"kernel": [launches, total_ms, algorithmic_bytes, units], ...} (bytes and
 * units are filled in for the sketch kernel: patterned bases read plus 16-byte
 * minimizer records written; and for the lookups: the record, its results
 * and the table words and offsets a probe reads) of
 * everything timed since the last
 * reset into buf (NUL-terminated) and returns 0, or returns the needed size
 * when cap is too small. Reading the report waits for the timed launches. */
void god_prof_enable(int on);
void god_prof_reset(void);
int god_prof_report(char *buf, uint64_t cap);
/* The timed launches since the last reset as a JSON list of [kernel, stream,
 * start_ms, end_ms] (streams numbered in order of appearance; times from an
 * event recorded on the default stream when timing was switched on or reset),
 * for seeing how launches on several streams overlap. Same return convention
 * as god_prof_report; at most 2^20 launches are kept. */
int god_prof_timeline(char *buf, uint64_t cap);

/* The batched sketch pass is captured into a CUDA graph per (shape, stream)
 * and replayed (on by default; calls on the legacy default stream launch
 * directly). 0 switches graphs off process-wide. */
void god_set_graphs(int on);

/* Autotuner table: JSON list of {"k","w","p","x","len_class","threads",
 * "chunks","ms"} entries chosen so far (god_params.tune = 1 fills it). Same
 * return convention as god_prof_report. */
int god_autotune_report(char *buf, uint64_t cap);

/* ----------------------------------------------------------------- serving
 * A continuous-batching server over one resident index: requests (read
 * batches) are queued, admitted into free slots while device memory allows,
 * merged with other waiting requests into one batched seeding pass, and run
 * concurrently on per-slot streams. Results are per-request host arrays.
 */
typedef struct god_server god_server;

typedef struct {
  int slots;               /* concurrent batches on the device (streams); default 4 */
  uint64_t mem_budget;     /* device bytes the server may hold for batches; 0 = 80% of free memory */
  uint64_t max_batch_bases;/* bases merged into one pass at most; default 64 Mi */
} god_server_config;

void god_server_config_init(god_server_config *c);
int god_server_create(const god_index *idx, const god_server_config *cfg, god_server **out);
/* Queues a request and returns its id. The reads and offsets stay in the
 * caller's host memory, which must remain valid and unchanged until
 * god_server_wait has returned for this request (the offsets are copied at
 * submit, the read bytes once, into the batch's pinned staging). */
int god_server_submit(god_server *s, const uint8_t *reads, const uint64_t *offsets, uint32_t n,
                      uint64_t *request_id);
/* Waits up to timeout_ms (negative = forever) for a request. On GOD_OK the
 * anchors (read_id local to the request) are returned as a host array
 * (release with god_free: a slice of the page-locked buffer that received its
 * batch's anchors, which returns to the server's pool once every slice of it
 * is freed, also after god_server_destroy) and, if latency_s is not NULL, the
 * time from submit to completion; GOD_EBUSY if it is not done in time. A
 * request that alone exceeds the memory budget completes with GOD_ENOMEM. */
int god_server_wait(god_server *s, uint64_t request_id, int timeout_ms, god_anchor **anchors,
                    uint64_t *n_anchors, double *latency_s);

typedef struct {
  uint64_t submitted, completed, batches, max_inflight_batches, merged_requests;
  uint64_t rejected;       /* requests larger than the memory budget */
  /* Seconds the worker threads spent, summed over slots: copying request
   * bytes into page-locked staging; allocating page-locked memory (staging
   * growth, result buffers); the device pass (input copy, seeding, with its
   * own synchronisations); cutting the result and copying it back. */
  double gather_s, pin_alloc_s, device_s, copy_back_s;
} god_server_stats;

int god_server_get_stats(god_server *s, god_server_stats *st);
int god_server_destroy(god_server *s);

#ifdef __cplusplus
}
#endif
#endif /* GOD_H */
