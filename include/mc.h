/*
 * mc.h -- C ABI of the GB300 (sm_103a) MetaCache-GPU hot path.
 *
 * MetaCache-GPU (Kobus et al., arXiv 2106.08150) classifies short DNA reads
 * against a database of reference genomes ("targets").  The database maps
 * minhash features of reference windows to the locations (target, window)
 * they occur in (Section 4.1); classification sketches each read, looks its
 * features up, accumulates the hit locations and labels the read by its top
 * candidate or by the lowest common ancestor (LCA) of the close candidates
 * in a taxonomy (Section 4.2).  Every step of both halves runs in CUDA
 * kernels of this library.
 *
 * Conventions for every function:
 *  - Return value: an mc_status code (MC_OK = 0).  On error a message is
 *    available from mc_last_error_string() (per calling thread).  No call
 *    traps or aborts; device-detected errors are written to a status word
 *    that the library reads back.
 *  - "device" pointers are CUDA global-memory pointers on the current
 *    device; "host" pointers are ordinary CPU memory.  Inputs are owned by
 *    the caller and only read during the call (stream-ordered for device
 *    inputs); outputs are caller-allocated.
 *  - Sequences are ASCII bytes; A/C/G/T in either case are bases, every
 *    other byte is an invalid base (Section 5.2 step 1: "N" and friends).
 *  - Streams are cudaStream_t values passed as void* (NULL = legacy stream).
 *
 * Build and query order: mc_db_create -> mc_db_add_targets (one or more
 * calls) -> mc_db_finalize -> mc_classify (any number of calls) ->
 * mc_db_free.  mc_db_add_targets after mc_db_finalize extends the database
 * (new targets get the next ids); the extension becomes visible to
 * mc_classify at the next mc_db_finalize.
 */
#ifndef MC_H
#define MC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MC_API_VERSION 2

/* Status codes returned by every entry point. */
typedef enum mc_status {
    MC_OK = 0,
    MC_ERR_ARG = 1,        /* invalid argument (range, null pointer, layout) */
    MC_ERR_STATE = 2,      /* call not allowed in the database's state */
    MC_ERR_OOM = 3,        /* device allocation failed or budget exceeded */
    MC_ERR_TABLE_FULL = 4, /* a table could not hold the data */
    MC_ERR_TIMEOUT = 5,    /* a bounded device wait gave up */
    MC_ERR_CUDA = 6,       /* a CUDA runtime call failed */
    MC_ERR_CAPACITY = 7    /* a size limit of this library was exceeded */
} mc_status;

#define MC_NO_TAXON 0xFFFFFFFFu  /* label of an unclassified read */
#define MC_NO_TARGET 0xFFFFFFFFu /* top target of a read without hits */

/* Limits of this implementation. */
#define MC_MAX_K 16               /* k-mers are packed in 32-bit words */
#define MC_MAX_SKETCH 32          /* one feature per lane of a warp */
#define MC_MAX_WINDOW_KMERS 512   /* w - k + 1 */
#define MC_MAX_CANDIDATES 8       /* m, top hits kept per read */
#define MC_MAX_QUERY_WINDOWS 64   /* windows of all mates of one query */
#define MC_MAX_QUERY_MATES 31     /* sequences (mates) of one query */
#define MC_MAX_INSERT 65536       /* largest max_insert */

typedef struct mc_db mc_db; /* opaque; owns every device allocation it makes */

/* Database parameters, fixed at mc_db_create (Section 5.2: defaults k = 16,
 * s = 16, window 127 with overlap k-1; the paper's GPU kernels also require
 * stride % 4 == 0 and w <= 128, which this library does not). */
typedef struct mc_db_params {
    uint32_t k;             /* k-mer length, 1..16 */
    uint32_t sketch_size;   /* s: features per window, 1..32 (Section 4.1) */
    uint32_t window_len;    /* w: bases per window, k..k+511 (Section 4.1) */
    uint32_t window_stride; /* distance of window starts, 1..w-k+1 (Section 4.1: w-k+1) */
    uint32_t bucket_cap;    /* locations kept per feature, 1..65535 (Section 4.1: 254);
                               the smallest (target, window) pairs are kept */
    uint32_t reserved;      /* must be 0 */
    uint64_t max_locations; /* optional capacity hint (0 = none) */
    uint64_t hbm_budget;    /* bytes the database may hold on the device (0 = no limit) */
} mc_db_params;

/* Classification parameters, per mc_classify call (Section 4.2). */
typedef struct mc_classify_params {
    uint32_t max_candidates; /* m: top hits kept, 1..8 (Section 4.2: usually 2..4) */
    uint32_t hits_min;       /* minimum top score to classify (Section 6.5: hit threshold) */
    uint32_t lca_band_pct;   /* 0..100: candidates with score >= (100-band)% of the top score
                                are "close"; one close candidate -> its taxon, several -> LCA */
    uint32_t max_insert;     /* read pairs: sliding-window span is max(len1+len2, max_insert);
                                0..MC_MAX_INSERT */
} mc_classify_params;

/* Device memory provider.  alloc returns device memory of at least `bytes`,
 * aligned to 256 bytes (as cudaMallocAsync and PyTorch's caching allocator
 * align), usable in stream order on `stream` (NULL on failure); free
 * releases it in stream order.  A block that is not 256-byte aligned is
 * handed back to free and the call fails with MC_ERR_OOM.  A provider such
 * as PyTorch's caching allocator can back every allocation of the
 * library. */
typedef struct mc_allocator {
    void* (*alloc)(void* ctx, size_t bytes, void* stream);
    void (*free)(void* ctx, void* ptr, size_t bytes, void* stream);
    void* ctx;
} mc_allocator;

/* Process-wide allocator (NULL restores the default, cudaMallocAsync /
 * cudaFreeAsync).  Set it before creating databases; a database frees its
 * memory with the allocator it was created with. */
int mc_set_allocator(const mc_allocator* allocator);

/* Creates an empty database.
 *  params : host; validated as documented in mc_db_params.
 *  n_taxa : number of taxonomy nodes (>= 1); taxon ids are 0..n_taxa-1.
 *  parent : host, n_taxa entries; parent[x] is x's parent, a root has
 *           parent[x] == x (NCBI-style tree, Section 4.1).  Cycles are
 *           rejected with MC_ERR_ARG.
 *  stream : stream for every build-side call of this database.
 *  out    : host; receives the handle.
 * The per-taxon lineage table used for constant-time LCA (Section 4.2) is
 * built on the device here.  Synchronises `stream`. */
int mc_db_create(const mc_db_params* params, uint32_t n_taxa, const uint32_t* parent, void* stream,
                 mc_db** out);

/* Adds targets (reference sequences) to the database (Section 4.1 build
 * phase, Section 5.2 build pipeline: encode, canonical k-mers, h1, sketch,
 * insert).
 *  n_targets : number of sequences in this call (may be 0).
 *  seq       : device, ASCII bases of all targets back to back.
 *  offs      : device, n_targets+1 byte offsets into seq, non-decreasing;
 *              target i is seq[offs[i] .. offs[i+1]).
 *  taxon     : host, n_targets taxon ids (< n_taxa, or MC_NO_TAXON).
 *  first_target_id : host out (nullable); ids are assigned densely in
 *              call order, so target i of this call gets *first + i.
 * Each target is cut into windows of window_len bases at multiples of
 * window_stride; window j of a target is location (target, j).  The inputs
 * are read before the call returns (synchronises the database stream).
 * MC_ERR_CAPACITY if the database would exceed 2^32-2 windows or 2^32-2
 * targets. */
int mc_db_add_targets(mc_db* db, uint32_t n_targets, const char* seq, const uint64_t* offs,
                      const uint32_t* taxon, uint32_t* first_target_id);

/* Publishes everything added so far in the condensed query layout
 * (Section 4.2 / 5.1: all buckets in one contiguous array, a single-value
 * hash table from feature to bucket).  Each feature keeps its bucket_cap
 * smallest locations, sorted ascending.  Idempotent; required before
 * mc_classify.  Synchronises the database stream.  MC_ERR_OOM if the sort
 * buffers cannot be allocated: nothing has changed and the call can be
 * repeated.  A failure after the sort has run (MC_ERR_OOM for the layout
 * buffers, MC_ERR_CUDA on a CUDA error, MC_ERR_TIMEOUT for a sort whose
 * tiles waited more than 2 s for earlier tiles' counts) keeps the previous
 * layout published for mc_classify, and later mc_db_add_targets and
 * mc_db_finalize calls return MC_ERR_STATE. */
int mc_db_finalize(mc_db* db);

/* ---------------------------------------------------------------------
 * Databases partitioned by target (Section 4.3: the reference targets are
 * split over several GPUs, each builds and queries a database of its own
 * targets, Section 4.2: and the top candidates of the partitions are
 * merged).  A shard holds a contiguous range of global target ids, given
 * in ascending order: shard 0 the first targets, shard 1 the next, and so
 * on.  The cap smallest locations of a feature over all targets are then
 * those of the earlier shards first, so shard s keeps at most
 * bucket_cap - prior(f) of its own locations of feature f, prior(f) being
 * f's locations in shards 0..s-1.  Built that way the shards together hold
 * exactly the database of all targets, and merged classification equals
 * the single-database result.  (The paper caps each partition on its own,
 * which keeps more locations than one database would; this library
 * enforces the single-database cap.)  Protocol: every shard adds its
 * targets, calls mc_db_feature_counts, the lists of the earlier shards are
 * exchanged (e.g. an all-gather), and each shard calls
 * mc_db_finalize_after with them; queries go to every shard
 * (mc_classify_debug with a cands buffer) and mc_merge_candidates merges
 * the lists. */

/* Features of the targets added so far (before the first finalize) and
 * how often each occurs, for the shards after this one: keys (device out,
 * max_keys entries) receives the features' keys in the library's internal
 * order (ascending; opaque values to pass to mc_db_finalize_after), counts
 * (device out) their location counts clamped to bucket_cap.  *n_keys
 * (host) = the number of features; MC_ERR_CAPACITY (nothing written) if it
 * exceeds max_keys.  Sorts the pending pairs in place (mc_db_finalize then
 * skips that sort).  MC_ERR_STATE after a finalize.  Synchronises the
 * database stream. */
int mc_db_feature_counts(mc_db* db, uint64_t max_keys, uint32_t* keys, uint32_t* counts, uint64_t* n_keys);

/* mc_db_finalize for a shard: the n_lists lists (host arrays of device
 * pointers keys[l], counts[l] and host sizes n_keys[l]; each from
 * mc_db_feature_counts of an earlier shard) give prior(f) = the sum of f's
 * counts, and feature f keeps at most max(0, bucket_cap - prior(f)) of this
 * database's locations.  With n_lists = 0 it is mc_db_finalize.
 * overflow_keys (mc_db_stats) counts the features whose locations here and
 * in the prior lists exceed bucket_cap.  Errors as mc_db_finalize. */
int mc_db_finalize_after(mc_db* db, uint32_t n_lists, const uint32_t* const* keys, const uint32_t* const* counts,
                         const uint64_t* n_keys);

/* Merges the top-m candidate lists of n_lists shards per query into the
 * global top m and labels each query exactly as mc_classify does.
 *  db         : any database with the taxonomy (its lineage table is used).
 *  params     : max_candidates = m of the lists; hits_min, lca_band_pct as
 *               for mc_classify (max_insert unused).
 *  cands      : host array of n_lists device pointers, each n_queries x m x
 *               {score, target, first window, last window} as written by
 *               mc_classify_debug (targets are the shard's local ids).
 *  target_base: host, n_lists global ids of each shard's target 0.
 *  taxon_of_target : device, n_targets taxa of the global targets.
 *  label, hits, top_target (nullable), cands_out (nullable, n_queries x m
 *  x 4, global targets): device outputs.
 * Synchronises `stream`. */
int mc_merge_candidates(const mc_db* db, const mc_classify_params* params, uint32_t n_queries, uint32_t n_lists,
                        const uint32_t* const* cands, const uint32_t* target_base, const uint32_t* taxon_of_target,
                        uint32_t n_targets, uint32_t* label, uint32_t* hits, uint32_t* top_target,
                        uint32_t* cands_out, void* stream);

/* Classifies queries (Section 4.2 query phase, Section 5.2 query steps 1-8).
 *  params    : host.
 *  n_seq     : number of sequences (mates) in seq.
 *  seq       : device, ASCII bases of all mates back to back.
 *  offs      : device, n_seq+1 byte offsets into seq (non-decreasing).
 *  n_queries : number of queries.
 *  qoffs     : device, n_queries+1 indices into the sequences: query q is
 *              mates qoffs[q] .. qoffs[q+1]-1 (1 = single-end, 2 = pair;
 *              all windows of all mates of a query form one hit list).
 *              At most MC_MAX_QUERY_MATES mates and MC_MAX_QUERY_WINDOWS
 *              windows per query (larger queries are left unclassified and
 *              reported by mc_classify_status).
 *  label     : device out, n_queries taxon ids or MC_NO_TAXON.
 *  hits      : device out, n_queries top scores (0 without hits).
 *  top_target: device out (nullable), n_queries target ids or MC_NO_TARGET.
 *  stream    : stream for this call.
 * Asynchronous: returns after enqueueing.  The call waits (on the device)
 * for the last mc_db_finalize.  Device-detected errors of a call are
 * reported by mc_classify_status.  The database must not be changed while
 * calls are in flight.
 * Reads of seq are made in whole 16-byte aligned chunks: the bytes of a
 * query's chunks that lie before its first or after its last base (at most
 * 15 on each side, never outside those aligned chunks) are read and
 * ignored. */
int mc_classify(const mc_db* db, const mc_classify_params* params, uint32_t n_seq, const char* seq,
                const uint64_t* offs, uint32_t n_queries, const uint32_t* qoffs, uint32_t* label,
                uint32_t* hits, uint32_t* top_target, void* stream);

/* Allocation-free classification (this library's addition; the paper has
 * no counterpart).  Same arguments, results, launch shape (the database's
 * tuning, mc_db_set_tuning) and asynchronous behaviour as mc_classify, for
 * callers that cannot allocate device memory during the
 * call -- for example a server whose GPU memory is entirely reserved by
 * another allocator, or a latency-critical loop that must avoid the
 * allocation path.  mc_classify takes its per-call scratch from the
 * allocator; this function allocates nothing and instead uses a fixed
 * scratch array of MC_NOALLOC_SCRATCH_BYTES compiled into the library,
 * which every GPU that loads the library holds until the process exits.
 *  - At most MC_NOALLOC_MAX_QUERIES queries per call; larger calls return
 *    MC_ERR_CAPACITY (split the batch).
 *  - The first call on each device looks up the device address of the
 *    scratch array (cudaGetSymbolAddress, with that device current); make
 *    that first call before any stream capture.  The address is kept for
 *    the life of the process: resetting the device (cudaDeviceReset) after
 *    that first call is not supported.
 *  - All calls on a device share the one scratch array: calls whose work
 *    overlaps on the GPU (other streams, other threads) race and corrupt
 *    each other.  Serialise them, e.g. on one stream.
 *  - Device-detected errors are reported by mc_classify_status as usual. */
#define MC_NOALLOC_MAX_QUERIES 16384u
#define MC_NOALLOC_SCRATCH_BYTES (48u << 20)
int mc_classify_noalloc(const mc_db* db, const mc_classify_params* params, uint32_t n_seq, const char* seq,
                        const uint64_t* offs, uint32_t n_queries, const uint32_t* qoffs, uint32_t* label,
                        uint32_t* hits, uint32_t* top_target, void* stream);

/* ---------------------------------------------------------------------
 * Batched classification of mixed-length query batches.
 *
 * The paper pushes reads through its GPU pipeline one batch at a time,
 * with memory allocated for one batch (Section 5.2), and bundles the
 * kernels of its segmented sort in a CUDA graph (Section 5.5).  Here a
 * whole set of batches -- each with its own buffers, read
 * lengths and single/paired mix -- goes through one set of kernel launches
 * (lookup, score, large path), or through one replay of a CUDA graph of
 * that launch set (mc_plan).  Results equal those of one mc_classify call
 * per batch, bit for bit. */

/* One batch of queries: the arguments of mc_classify for one call. */
typedef struct mc_batch {
    uint32_t n_seq;          /* sequences (mates) of the batch */
    uint32_t n_queries;      /* queries of the batch */
    const char* seq;         /* device, ASCII bases of all mates */
    const uint64_t* offs;    /* device, n_seq+1 byte offsets into seq */
    const uint32_t* qoffs;   /* device, n_queries+1 mate indices (as in mc_classify) */
    uint32_t* label;         /* device out, n_queries */
    uint32_t* hits;          /* device out, n_queries */
    uint32_t* top_target;    /* device out, n_queries (nullable) */
} mc_batch;

/* Launch shape of the classification kernels.  Every setting gives the same
 * results; only the speed differs.  Zero fields take the defaults.
 *  score_mode  : how a query's gathered locations are counted and scored
 *                (the paper's segmented sort, Section 5.5, and window
 *                scoring, Section 5.6): 1 = sort path (default): one warp
 *                gathers the query's locations into registers and sorts
 *                them; 2 = hash path: per-warp hash histogram in shared
 *                memory.  The sort path needs 32-bit locations (mc_db_stats
 *                loc_bytes == 4) and histogram keys of that width
 *                (wide_keys 0); otherwise the hash path is used.
 *  sort_max    : sort path: largest number of gathered locations a query
 *                may have to be sorted, 256, 512, 1024 (default) or 2048; each
 *                size class up to it has its own kernel; larger queries go
 *                to the hash path's medium and large kernels.
 *  hist_slots  : hash path: shared-memory histogram slots per query: 256,
 *                512 (default) or 1024.  Queries whose distinct locations
 *                do not fit go to the medium (2,048 slots) and large paths.
 *  probe_batch : feature-table probes in flight per lane (32 lanes probe
 *                together): 2 (default), 4 or 8.
 *  gather_batch: hash path: bucket-location loads in flight per lane: 4, 8
 *                (default) or 16.
 *  lookup_warps: warps per CTA of the lookup kernel: 4 or 8 (default).
 *  score_warps : warps per CTA of the hash path's score kernel: 2 or 4 (default).
 *  wide_keys   : 0 (default) = the shared-memory histograms key a location
 *                by 32 bits (target << b | window) when every target and
 *                window id of the database fits 32 bits, else by 64; 1 =
 *                always 64-bit keys (hash path).
 * One warp carries one query in every kernel. */
typedef struct mc_tuning {
    uint32_t hist_slots;
    uint32_t probe_batch;
    uint32_t gather_batch;
    uint32_t lookup_warps;
    uint32_t score_warps;
    uint32_t wide_keys;
    uint32_t score_mode;
    uint32_t sort_max;
} mc_tuning;

/* Sets the launch shape used by later classify calls on this database that
 * take no explicit tuning (mc_classify, mc_classify_batches with NULL).
 * NULL restores the defaults.  MC_ERR_ARG for a value outside the sets
 * above. */
int mc_db_set_tuning(mc_db* db, const mc_tuning* tuning);

/* Classifies n_batches batches (host array of descriptors; device buffers)
 * in one launch set on `stream`.  tuning: NULL = the database's.  Per-batch
 * limits as in mc_classify; the total query count must be below 2^32.
 * Asynchronous; errors as mc_classify (mc_classify_status). */
int mc_classify_batches(const mc_db* db, const mc_classify_params* params, const mc_tuning* tuning,
                        uint32_t n_batches, const mc_batch* batches, void* stream);

/* A reusable classification plan: scratch memory for up to max_queries
 * queries in up to max_batches batches, and a CUDA graph of the whole
 * launch set, captured once.  mc_plan_run replays the graph for a new set
 * of batches: it copies the batch descriptors (host, n_batches) to the
 * device and launches the graph on `stream`.  A plan is re-captured
 * automatically when its database has been finalized again since.  Runs of
 * one plan are serialised (a run waits on the host for the previous run's
 * descriptor copy).  MC_ERR_CAPACITY if a run exceeds max_batches or
 * max_queries.  mc_plan_free synchronises and releases the plan. */
typedef struct mc_plan mc_plan;
int mc_plan_create(const mc_db* db, const mc_classify_params* params, const mc_tuning* tuning,
                   uint32_t max_batches, uint32_t max_queries, mc_plan** out);
int mc_plan_run(mc_plan* plan, uint32_t n_batches, const mc_batch* batches, void* stream);
int mc_plan_kernels(const mc_plan* plan);  /* kernel launches per run (graph kernel nodes) */
void mc_plan_free(mc_plan* plan);

/* Autotuner: times every lookup setting (probe_batch x lookup_warps) and
 * every score setting (the hash path's hist_slots x gather_batch x
 * score_warps, and, for databases with 32-bit locations, the sort path's
 * sort_max, each with the medium and large paths it leaves) on the given
 * sample batches (at most 2^20 queries
 * in total), `reps` times each, and writes the fastest setting to *best.
 * If `times` is not NULL it receives up to max_times records
 * {setting, kernel ms (mean over reps)} in the order tried; *n_times (if
 * not NULL) the number tried.  Synchronises the database stream. */
typedef struct mc_tuning_time {
    mc_tuning tuning;
    uint32_t stage;  /* 0 = lookup setting, 1 = score setting */
    float ms;
} mc_tuning_time;
int mc_autotune(const mc_db* db, const mc_classify_params* params, uint32_t n_batches, const mc_batch* batches,
                uint32_t reps, mc_tuning* best, mc_tuning_time* times, uint32_t max_times, uint32_t* n_times);

/* ---------------------------------------------------------------------
 * Served classification: a resident database and a request loop.
 *
 * The paper holds a database in memory for an interactive session of
 * successive queries (Section 4) and queries a database straight after its
 * build (on-the-fly mode, Section 6.3).  mc_server runs that as a service
 * whose database also grows while it serves: jobs (host buffers) arrive at any time from any thread; a
 * scheduler thread inside the library admits them while their device
 * memory fits the server's HBM limit, and packs the admitted jobs into
 * launch sets (continuous batching: jobs that arrive while earlier sets
 * are on the GPU go into the next set, on the next of n_streams streams,
 * so copies and kernels of consecutive sets overlap).  Each launch set is
 * one replay of a classification plan (mc_plan).  Extensions (new
 * genomes) are applied between launch sets.  Every job is classified
 * against one database state (epoch): a job split over several launch
 * sets delays a pending extension until its last piece is enqueued, a job
 * submitted after an extension request runs after that extension, and
 * launch sets in flight keep reading the state they were enqueued
 * against while an extension replaces it. */

typedef struct mc_server mc_server;

typedef struct mc_server_config {
    uint32_t n_streams;          /* launch sets in flight at once (0 = 2) */
    uint32_t max_set_queries;    /* queries per launch set (0 = 2^21); larger jobs are split */
    uint32_t max_set_jobs;       /* job pieces per launch set (0 = 256) */
    uint32_t reserved;
    uint64_t hbm_limit;          /* device bytes the server may hold for job buffers
                                    (0 = half of the free memory at creation) */
} mc_server_config;

/* A classification job.  All buffers are on the host and must stay valid
 * (and the outputs unread) until mc_server_wait reports the job done.
 * Page-locked host memory lets the copies run asynchronously; pageable
 * memory is copied synchronously by the scheduler thread. */
typedef struct mc_job {
    uint32_t n_seq;          /* sequences (mates) */
    uint32_t n_queries;      /* queries */
    const char* seq;         /* host, ASCII bases */
    const uint64_t* offs;    /* host, n_seq+1 */
    const uint32_t* qoffs;   /* host, n_queries+1 (as in mc_classify) */
    uint32_t* label;         /* host out, n_queries */
    uint32_t* hits;          /* host out, n_queries */
    uint32_t* top_target;    /* host out, n_queries (nullable) */
} mc_job;

/* Timing and state of a finished job (seconds since server creation). */
typedef struct mc_job_info {
    double t_submit, t_launch, t_done;
    uint64_t epoch;          /* database epoch the job was classified against */
    uint32_t pieces;         /* launch sets the job was split over */
    int status;              /* MC_OK, or the error of the job */
} mc_job_info;

typedef struct mc_server_stats {
    uint64_t jobs_submitted, jobs_done, queries_done, launch_sets, extensions;
    uint64_t epoch;              /* database epoch now */
    uint64_t hbm_in_use, hbm_limit, hbm_peak;
    double p50_latency_s, p99_latency_s, max_latency_s;  /* over finished jobs */
    double busy_s;               /* from the first submission to the last completion */
    double extension_mean_s, extension_max_s;  /* time of an applied extension (add + finalize,
                                                  database stream idle at both ends) */
} mc_server_stats;

/* Creates a server over a finalized database.  The server owns the
 * database's use from then on: the caller makes no other call on `db`
 * until mc_server_free (which does not free the database). */
int mc_server_create(mc_db* db, const mc_classify_params* params, const mc_server_config* config,
                     mc_server** out);

/* Queues a job (non-blocking) and returns its id.  MC_ERR_OOM if the job
 * alone needs more device memory than the server's limit. */
int mc_server_submit(mc_server* srv, const mc_job* job, uint64_t* job_id);

/* Queues the insertion of new targets (host buffers, copied before the
 * call returns; taxon ids as in mc_db_add_targets).  The scheduler adds
 * and finalizes them between launch sets.  *first_target_id receives the
 * id of the first new target. */
int mc_server_extend(mc_server* srv, uint32_t n_targets, const char* seq, const uint64_t* offs,
                     const uint32_t* taxon, uint32_t* first_target_id);

/* Waits up to timeout_s seconds (< 0: forever) for a job.  MC_OK and
 * *info (nullable) when it is done (the job's own error is info->status);
 * MC_ERR_TIMEOUT if it is not done yet; MC_ERR_ARG for an unknown id.
 * A job's record is dropped after the first successful wait. */
int mc_server_wait(mc_server* srv, uint64_t job_id, double timeout_s, mc_job_info* info);

/* Waits until every queued job and extension is done (timeout as above). */
int mc_server_drain(mc_server* srv, double timeout_s);

int mc_server_stats_get(mc_server* srv, mc_server_stats* out);

/* Drains, stops the scheduler and releases the server's resources. */
void mc_server_free(mc_server* srv);

/* Synchronises `stream` and returns (and clears) the first device-detected
 * error of earlier mc_classify calls of this database (MC_ERR_CAPACITY for
 * a query with more distinct hit locations than the largest per-query
 * histogram holds, or more windows than MC_MAX_QUERY_WINDOWS). */
int mc_classify_status(const mc_db* db, void* stream);

/* Releases the database and all its device memory (synchronises its stream). */
void mc_db_free(mc_db* db);

/* Writes the finalized database to a file (Section 4.1: the database and
 * the taxonomy are written to the file system after the build; Section 4.2:
 * a saved database is loaded in the condensed layout).  The file holds the
 * parameters, the taxonomy (parent array), the targets' taxa and window
 * bases, the location array and the feature table.  MC_ERR_STATE if
 * additions are pending (call mc_db_finalize first); MC_ERR_ARG if the
 * file cannot be written.  Synchronises the database stream. */
int mc_db_save(const mc_db* db, const char* path);

/* Reads a database written by mc_db_save into a new handle (device memory
 * from the current allocator, build-side calls on `stream`).  The loaded
 * database can be classified against at once and extended like any other.
 * MC_ERR_ARG if the file is missing, truncated or not a database of this
 * format version. */
int mc_db_load(const char* path, void* stream, mc_db** out);

/* ---------------------------------------------------------------------
 * Inspection and test exports.
 * ------------------------------------------------------------------- */

typedef struct mc_db_stats_t {
    uint64_t n_targets;
    uint64_t n_windows;         /* all windows of all targets */
    uint64_t n_pairs;           /* (feature, location) pairs offered */
    uint64_t n_keys;            /* distinct features */
    uint64_t n_locations;       /* locations stored after the cap */
    uint64_t overflow_keys;     /* features that had more than bucket_cap locations (after a
                                   live extension: counted over the kept locations of the
                                   earlier targets plus those of the new ones) */
    uint64_t dropped_locations; /* n_pairs - n_locations */
    uint64_t table_slots;       /* slots of the feature table (8 bytes each) */
    uint64_t max_probe;         /* longest probe distance in the feature table */
    uint64_t device_bytes;      /* bytes held on the device */
    double load_factor;         /* n_keys / table_slots */
    uint32_t finalized;         /* 1 if no additions are pending */
    uint32_t max_depth;         /* deepest taxonomy level */
    uint32_t loc_bytes;         /* bytes per stored location: 4 when every (target, window)
                                   fits 32 bits as target << b | window, else 8 */
    uint32_t reserved;
} mc_db_stats_t;

/* Fills *out (host) with the database's counters (no synchronisation). */
int mc_db_stats(const mc_db* db, mc_db_stats_t* out);

/* Canonical dump of the finalized database: features f with
 * key_lo <= f < key_hi in ascending order, each with its bucket in
 * ascending order.  Host outputs: keys[n], counts[n], locs (concatenated
 * buckets, (target << 32) | window).  If more than max_keys features or
 * max_locs locations qualify, nothing is written and MC_ERR_CAPACITY is
 * returned with *n_keys / *n_locs set to the required sizes.
 * Synchronises the database stream. */
int mc_db_dump(const mc_db* db, uint64_t key_lo, uint64_t key_hi, uint64_t max_keys, uint64_t max_locs,
               uint32_t* keys, uint32_t* counts, uint64_t* locs, uint64_t* n_keys, uint64_t* n_locs);

/* Window layout of sequences (Section 4.1): win_offs (device out, n_seq+1)
 * receives the exclusive prefix sum of ceil((L-k+1)/stride) (0 if L < k).
 * Asynchronous on `stream`. */
int mc_window_offsets(const mc_db_params* params, uint32_t n_seq, const uint64_t* offs, uint64_t* win_offs,
                      void* stream);

/* Minhash sketches of every window (Section 2, Section 5.2 steps 1-3):
 * sketch[w * sketch_size + i] (device out) = i-th smallest distinct h1
 * value of window w's valid canonical k-mers, 0 past counts[w] (device
 * out, n_windows).  win_offs from mc_window_offsets; n_windows =
 * win_offs[n_seq].  Asynchronous on `stream`. */
int mc_sketch(const mc_db_params* params, uint32_t n_seq, const char* seq, const uint64_t* offs,
              const uint64_t* win_offs, uint64_t n_windows, uint32_t* sketch, uint32_t* counts,
              void* stream);

/* mc_classify with test outputs.  cands (device out, nullable):
 * n_queries x max_candidates x {score, target, first window, last window}
 * of the top candidates (unused slots: score 0, target MC_NO_TARGET).
 * counters (device out, nullable, MC_DEBUG_COUNTERS x uint64, accumulated):
 * [0] features looked up, [1] locations gathered, [2] distinct locations,
 * [3] queries sent to the large-histogram path, [4] features found, [5]
 * 32-byte sectors of the gathered buckets, [6] queries finished on the
 * medium-histogram path; then per scoring kernel k (0 hash-path score
 * kernel, 1-3 sort path for up to 256/512/1024 locations, 4 medium path,
 * 5 large path, 6 sort path for up to 2048 locations): [7 + 3k] queries it
 * finished, [8 + 3k] their found features, [9 + 3k] their 32-byte
 * sectors. */
#define MC_DEBUG_COUNTERS 28
int mc_classify_debug(const mc_db* db, const mc_classify_params* params, uint32_t n_seq, const char* seq,
                      const uint64_t* offs, uint32_t n_queries, const uint32_t* qoffs, uint32_t* label,
                      uint32_t* hits, uint32_t* top_target, uint32_t* cands, uint64_t* counters,
                      void* stream);

/* ---------------------------------------------------------------------
 * Tracing and launch accounting (no counterpart in the paper beyond its
 * per-stage breakdown, Section 6.4).
 * ------------------------------------------------------------------- */

/* Enables (1) or disables (0) tracing: each kernel launch of the library is
 * bracketed by CUDA events recorded on the stream it is launched on. */
int mc_trace_enable(int on);

/* Synchronises the recorded events and writes one line per kernel,
 * "name launches total_ms", to buf (host, NUL-terminated, truncated to
 * len).  Returns the number of bytes the full report needs (excluding the
 * NUL).  reset != 0 clears the accumulated times afterwards. */
int mc_trace_report(char* buf, size_t len, int reset);

/* Number of kernel launches the library has issued in this process. */
uint64_t mc_kernel_launches(void);

/* Test export: arms a one-shot stall of the next database sort in this
 * process (any database), to exercise the bounded wait of its single-pass
 * radix sort (decoupled look-back: each tile of 4,096 pairs waits for the
 * digit counts of the tiles before it).  The last of the sort's four passes
 * then skips its first tile, whose counts are therefore never published;
 * the next tile's wait gives up after limit_ns (1e6..2e9) and the
 * mc_db_finalize that ran the sort fails with MC_ERR_TIMEOUT, keeping the
 * previous layout published (as documented there).  Every write of the
 * disturbed pass stays inside its buffer.  If the last pass has fewer than
 * two tiles the stall is dropped and the sort runs normally.  MC_ERR_ARG
 * for a limit outside the range. */
int mc_debug_stall_next_sort(uint64_t limit_ns);

/* Message of the last error on the calling thread ("" if none). */
const char* mc_last_error_string(void);

/* Name of a status code. */
const char* mc_status_string(int status);

/* MC_API_VERSION of the loaded library. */
int mc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MC_H */
