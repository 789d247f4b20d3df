// Internal interface between the translation units of libmc (host side).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/mc.h"
#include "mc_common.cuh"

namespace mc {

// Launch accounting and optional per-kernel event tracing (mc_api.cu).
void note_launch(cudaStream_t s);  // not counted while `s` is being captured
void note_launches(uint64_t n);     // kernels of a graph replay
struct TraceScope {
    int slot = -1;
    cudaStream_t stream = nullptr;
    TraceScope(const char* name, cudaStream_t s);
    ~TraceScope();
};
#define MC_LAUNCH(name, stream, ...)                \
    do {                                            \
        ::mc::TraceScope trace_scope_((name), (stream)); \
        __VA_ARGS__;                                \
        ::mc::note_launch(stream);                  \
    } while (0)

// Device memory through the database's allocator (stream-ordered).
struct Mem {
    mc_allocator a;
    void* alloc(size_t bytes, cudaStream_t s) const;
    void free(void* p, size_t bytes, cudaStream_t s) const;
};

// A scoped temporary device buffer, freed in stream order.
template <class T>
struct Tmp {
    const Mem* mem = nullptr;
    cudaStream_t stream = nullptr;
    T* ptr = nullptr;
    size_t bytes = 0;
    Tmp() = default;
    Tmp(const Mem& m, size_t n, cudaStream_t s) : mem(&m), stream(s), bytes(n * sizeof(T)) {
        ptr = bytes ? static_cast<T*>(m.alloc(bytes, s)) : nullptr;
    }
    Tmp(const Tmp&) = delete;
    Tmp& operator=(const Tmp&) = delete;
    ~Tmp() {
        if (ptr) mem->free(ptr, bytes, stream);
    }
    bool ok() const { return bytes == 0 || ptr != nullptr; }
    T* release() {
        T* p = ptr;
        ptr = nullptr;
        return p;
    }
};

// ------------------------------------------------------------ mc_build.cu
// Exclusive prefix sum of n u64 values into out[0..n); out[n] = total.
// in may alias out.
cudaError_t scan_exclusive_sum(const Mem& mem, const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t s);

// win_offs[i] = exclusive prefix of windows per sequence, win_offs[n] =
// total.  Sets *bad_offs (device) if offs decreases.
cudaError_t window_offsets(const Mem& mem, const SketchParams& p, uint32_t n_seq, const uint64_t* offs,
                           uint64_t* win_offs, uint32_t* bad_offs, cudaStream_t s);

// Debug sketch export (mc_sketch).
cudaError_t sketch_windows(const SketchParams& p, uint32_t n_seq, const uint8_t* seq, const uint64_t* offs,
                           const uint64_t* win_offs, uint64_t n_windows, uint32_t* sketch, uint32_t* counts,
                           cudaStream_t s);

// Build: sketch every window of the call's targets and write its (h2(f) <<
// 32 | global window) pairs to pairs[lw * s + i] (sentinel past the
// sketch).  *real_pairs (device) += pairs written.
cudaError_t emit_pairs(const SketchParams& p, uint32_t n_targets, const uint8_t* seq, const uint64_t* offs,
                       const uint64_t* win_offs, uint64_t n_windows, uint32_t gw_base, uint64_t* pairs,
                       unsigned long long* real_pairs, cudaStream_t s);

// Stable LSD radix sort of pairs by their upper 32 bits (4 passes of 8
// bits).  The first pass drops sentinel pairs.  in holds n_total entries
// on entry, the n_real sorted real pairs on return; tmp has n_total room.
// Synchronizes the stream; cudaErrorMemoryAllocation (before any pair is
// touched) if its scratch cannot be allocated; cudaErrorTimeout if a tile's
// wait for earlier tiles' counts gave up (the order is then wrong).
cudaError_t sort_pairs(const Mem& mem, uint64_t* in, uint64_t* tmp, uint64_t n_total, uint64_t n_real,
                       cudaStream_t s);
// Arms a one-shot stall of the next sort_pairs call's last pass (a test of
// the bounded look-back wait): that pass skips its tile 0, so tile 1 waits
// for counts that are never published and gives up after limit_ns; the sort
// then returns cudaErrorTimeout.  Dropped (the sort runs normally) when the
// last pass has fewer than two tiles.
void arm_sort_stall(uint64_t limit_ns);

struct FinalizeOut {
    uint64_t n_keys = 0;
    uint64_t n_kept = 0;
    uint64_t overflow_keys = 0;
    void* locs = nullptr;        // n_kept locations (encoding: loc_bytes)
    uint64_t* table = nullptr;   // table_len packed words (TableFmt)
    uint64_t table_len = 0;
    uint64_t table_bytes = 0;
    TableFmt fmt{1, 1};
    uint32_t max_probe = 0;
    bool table_full = false;     // no table format can hold the layout
};

// Location encoding of a database: jbits > 0 = 32-bit words target << jbits
// | window (every target and window id fits; the all-ones word is never a
// location), 0 = 64-bit words target << 32 | window.
__host__ __device__ inline uint32_t loc_bytes(uint32_t jbits) { return jbits ? 4u : 8u; }

// Condensed layout from sorted pairs: keep the first `cap` pairs of each
// feature, convert global windows to (target, window) locations in the
// jbits encoding, build the ordered linear-probing feature table.  wbase:
// n_targets+1 global window bases.
cudaError_t finalize_pairs(const Mem& mem, const uint64_t* sorted, uint64_t n, uint32_t cap, const uint32_t* wbase,
                           uint32_t n_targets, uint32_t jbits, FinalizeOut* out, cudaStream_t s);

// c[0..na+nb) = the merge of the sorted pair runs a and b (ties from a).
cudaError_t merge_sorted_pairs(const uint64_t* a, uint64_t na, const uint64_t* b, uint64_t nb, uint64_t* c,
                               cudaStream_t s);

// Sharded builds (Section 4.3): distinct features of sorted pairs a[0..n)
// (h2 keys ascending) with their counts clamped to cap; *n_keys = the
// number of features, written only when they fit max.
cudaError_t feature_counts(const Mem& mem, const uint64_t* a, uint64_t n, uint32_t cap, uint64_t max, uint32_t* keys,
                           uint32_t* counts, uint64_t* n_keys, cudaStream_t s);
// Turns into sentinels, in sorted pairs a[0..n), the pairs each feature
// gives up to earlier shards: feature f keeps at most cap - prior(f) pairs,
// prior(f) = the sum of f's counts in the n_lists device lists (keys
// ascending, host arrays of device pointers).  *overflow = features whose
// pairs together with the prior ones exceed cap (features without prior
// pairs are left to the plain cap of finalize_pairs).
cudaError_t apply_prior(const Mem& mem, uint64_t* a, uint64_t n, uint32_t cap, uint32_t n_lists,
                        const uint32_t* const* keys, const uint32_t* const* counts, const uint64_t* list_n,
                        uint64_t* overflow, cudaStream_t s);

// The (h2 << 32 | global window) pairs of a finalized layout, in layout
// order (out has n_kept entries).
cudaError_t reconstruct_pairs(const uint64_t* table, uint64_t table_len, TableFmt fmt, const void* locs, uint32_t jbits,
                              const uint32_t* wbase, uint64_t* out, cudaStream_t s);

// Taxonomy: depth per node and lineage rows lin[x * stride + d].
cudaError_t taxonomy_depths(const uint32_t* parent, uint32_t n_taxa, uint32_t* depth, uint32_t* max_depth,
                            uint32_t* cycle_flag, cudaStream_t s);
cudaError_t taxonomy_lineage(const uint32_t* parent, uint32_t n_taxa, const uint32_t* depth, uint32_t* lin,
                             uint32_t stride, cudaStream_t s);

// Dump support: entries of the table whose feature is in [lo, hi), and
// their buckets as 64-bit locations (target << 32 | window).
cudaError_t dump_select(const uint64_t* table, uint64_t table_len, TableFmt fmt, uint64_t lo, uint64_t hi,
                        uint32_t* keys, uint64_t* offs, uint32_t* counts, uint64_t cap, unsigned long long* n_sel,
                        cudaStream_t s);
cudaError_t dump_gather(const void* locs, uint32_t jbits, const uint64_t* src_off, const uint32_t* counts,
                        const uint64_t* dst_off, uint64_t n, uint64_t* out, cudaStream_t s);

// --------------------------------------------------------- mc_classify.cu
struct ClassifyDb {
    const uint64_t* table;  // packed feature-table words
    TableFmt fmt;
    uint32_t max_probe;
    const void* locs;       // locations, 32-bit words when jbits > 0, else 64-bit
    const uint32_t* taxon_of_target;
    uint32_t n_targets;
    const uint32_t* lineage;
    const uint32_t* depth;
    uint32_t lin_stride;
    uint32_t n_taxa;
    SketchParams sp;
    // > 0: every (target, window) of the database fits 32 bits as
    // target << jbits | window without being all ones: the locations are
    // stored in that form and the histograms can key by it; 0: 64-bit
    uint32_t jbits;
};

// jbits for a database of n_targets targets with at most max_windows
// windows each (0 when target and window ids do not fit 32 bits together).
uint32_t compact_key_bits(uint64_t n_targets, uint64_t max_windows);

// One batch of a multi-batch launch: the device pointers of an mc_batch.
struct BatchDesc {
    const uint8_t* seq;
    const uint64_t* offs;
    const uint32_t* qoffs;
    uint32_t* label;
    uint32_t* hits;
    uint32_t* top_target;
};

struct ClassifyQuery {
    // single batch (batches == nullptr)
    const uint8_t* seq;
    const uint64_t* offs;
    const uint32_t* qoffs;
    uint32_t n_q;  // queries; in the multi-batch form the capacity the scratch was sized for
    uint32_t m, hits_min, band, max_insert;
    uint32_t* label;
    uint32_t* hits;
    uint32_t* top_target;
    uint32_t* cands;  // indexed by query number (over all batches)
    unsigned long long* counters;
    uint32_t* status;
    // multi-batch form: bhdr (device) = {number of batches B, total queries,
    // then the B + 1 entry exclusive prefix of the batches' query counts};
    // query q of the launch is query q - prefix[b] of the batch b holding it
    const BatchDesc* batches = nullptr;
    const uint32_t* bhdr = nullptr;
};

// Launch shape of the classification kernels (mc_tuning).
constexpr uint32_t SCORE_SORT = 1, SCORE_HASH = 2;
struct Tuning {
    uint32_t hist_slots, probe_batch, gather_batch, lookup_warps, score_warps, wide_keys, score_mode, sort_max;
};
constexpr Tuning DEFAULT_TUNING{512, 2, 8, 8, 4, 0, SCORE_SORT, 1024};
bool tuning_valid(const Tuning& t);

// Device scratch of one classify launch set for up to n_q_cap queries.
struct ClassifyScratch {
    uint32_t* ovf;         // large-path queue (n_q_cap) + queue counters
    uint4* meta;           // per query of a chunk
    uint32_t* mid;         // medium-path queue of a chunk
    uint64_t* glist;       // bucket lists of a chunk
    unsigned char* large;  // large-path working memory
    uint32_t n_q_cap, chunk, large_warps;
};
uint32_t classify_default_large_warps();
size_t classify_scratch_bytes(uint32_t n_q_cap, uint32_t sketch_size, uint32_t large_warps);
ClassifyScratch classify_scratch_carve(unsigned char* base, uint32_t n_q_cap, uint32_t sketch_size,
                                       uint32_t large_warps);

// Enqueues one launch set (queue reset, lookup + score per chunk, large
// path) on `s`; no allocation, no synchronisation, so it can be captured
// in a CUDA graph.  *n_kernels (nullable) receives the kernel launches.
cudaError_t classify_enqueue(const ClassifyDb& db, const ClassifyQuery& q, const Tuning& t,
                             const ClassifyScratch& sc, cudaStream_t s, int* n_kernels);

// Allocates the scratch for q.n_q queries from `mem` and enqueues.
cudaError_t classify_launch(const Mem& mem, const ClassifyDb& db, const ClassifyQuery& q, const Tuning& t,
                            cudaStream_t s);

// Timing of one launch-shape candidate (autotuner).
struct TuneRecord {
    Tuning t;
    uint32_t stage;  // 0 lookup, 1 score + large path
    float ms;
};
// Times every lookup and score setting on the queries of q (at most one
// chunk), reps runs each; returns the fastest setting.  Synchronises `s`.
cudaError_t classify_autotune(const ClassifyDb& db, const ClassifyQuery& q, const ClassifyScratch& sc,
                              uint32_t reps, cudaStream_t s, Tuning* best, std::vector<TuneRecord>* records);
constexpr uint32_t CLASSIFY_CHUNK = 1u << 20;  // queries per lookup/score round

// Classification that allocates nothing: every scratch buffer is carved out
// of `scratch` (scratch_len bytes, 256-byte aligned).  classify_noalloc_bytes
// is the size a call with n_q queries needs.
size_t classify_noalloc_bytes(uint32_t n_q, uint32_t sketch_size);
cudaError_t classify_launch_noalloc(const ClassifyDb& db, const ClassifyQuery& q, const Tuning& t,
                                   unsigned char* scratch, size_t scratch_len, cudaStream_t s);

// One shard's top-m lists (device, n_q x m x {score, target, j0, j1}) and
// the global id of its target 0.
struct MergeList {
    const uint32_t* cands;
    uint32_t base;
};
// Merges n_lists shards' top-m lists per query and labels the result
// (taxon: device, n_targets global targets).  Synchronises `s`.
cudaError_t merge_candidates(const Mem& mem, const ClassifyDb& db, const uint32_t* taxon, uint32_t n_targets,
                             const MergeList* lists, uint32_t n_lists, uint32_t n_q, uint32_t m, uint32_t hits_min,
                             uint32_t band, uint32_t* label, uint32_t* hits, uint32_t* top_target, uint32_t* cands_out,
                             cudaStream_t s);

// ------------------------------------------------------------- mc_api.cu
// Records an error message for mc_last_error_string and returns `code`.
int report_error(int code, const char* fmt, ...);
// Checks a classify call and fills the kernel views of the database and the
// query (no allocation); makes `stream` wait for the last finalize.
int classify_prepare(const mc_db* db, const mc_classify_params* params, const char* seq, const uint64_t* offs,
                     uint32_t n_queries, const uint32_t* qoffs, uint32_t* label, uint32_t* hits,
                     uint32_t* top_target, cudaStream_t stream, ClassifyDb* cdb, ClassifyQuery* q);
// Records that classify work on `stream` reads the database's current
// layout (a later finalize frees that layout only after this work).
int classify_done(const mc_db* db, cudaStream_t stream);
// The launch shape later classify calls of the database use (mc_db_set_tuning).
Tuning db_tuning(const mc_db* db);

}  // namespace mc
