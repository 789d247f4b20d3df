// C ABI of the library (include/mc.h): argument checking, device memory
// ownership and the orchestration of the build and query kernels.  Every
// step of the method itself runs in the kernels of mc_build.cu and
// mc_classify.cu; this file only validates, allocates, copies metadata and
// launches.
#include <algorithm>
#include <atomic>
#include <string>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "mc_internal.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear sticky-free errors
    if (e == cudaErrorMemoryAllocation) return fail(MC_ERR_OOM, "%s: out of device memory", what);
    if (e == cudaErrorTimeout) return fail(MC_ERR_TIMEOUT, "%s: a bounded device wait gave up", what);
    return fail(MC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define MC_CU(call)                                   \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

void* default_alloc(void*, size_t bytes, void* stream) {
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void default_free(void*, void* p, size_t, void* stream) { cudaFreeAsync(p, (cudaStream_t)stream); }

std::mutex g_alloc_mu;
mc_allocator g_alloc = {default_alloc, default_free, nullptr};
bool g_pool_configured = false;

// Keep freed blocks of the default stream-ordered pool instead of returning
// them to the driver at every synchronisation (per-call scratch is reused).
void configure_default_pool() {
    if (g_pool_configured) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    g_pool_configured = true;
}

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

}  // namespace

namespace {
// ---- launch accounting and tracing
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_trace_on{0};
std::mutex g_trace_mu;
struct TraceRec {
    const char* name;
    cudaEvent_t a, b;
};
std::vector<TraceRec> g_trace_pending;
struct TraceAcc {
    uint64_t n = 0;
    double ms = 0;
};
std::vector<std::pair<std::string, TraceAcc>> g_trace_acc;
}  // namespace

namespace mc {
bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return st != cudaStreamCaptureStatusNone;
}

void note_launch(cudaStream_t s) {
    if (!capturing(s)) g_launches.fetch_add(1, std::memory_order_relaxed);
}

void note_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

TraceScope::TraceScope(const char* name, cudaStream_t s) : stream(s) {
    if (!g_trace_on.load(std::memory_order_relaxed) || capturing(s)) return;
    TraceRec r{name, nullptr, nullptr};
    if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    cudaEventRecord(r.a, s);
    std::lock_guard<std::mutex> lock(g_trace_mu);
    slot = (int)g_trace_pending.size();
    g_trace_pending.push_back(r);
}

TraceScope::~TraceScope() {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lock(g_trace_mu);
    if (slot < (int)g_trace_pending.size()) cudaEventRecord(g_trace_pending[slot].b, stream);
}

// Kernels use 16- and 32-byte vector accesses from the start of a block:
// a provider's block must be 256-byte aligned (else it is returned).
void* Mem::alloc(size_t bytes, cudaStream_t s) const {
    void* p = a.alloc(a.ctx, bytes, (void*)s);
    if (p && ((uintptr_t)p & 255u)) {
        a.free(a.ctx, p, bytes, (void*)s);
        return nullptr;
    }
    return p;
}
void Mem::free(void* p, size_t bytes, cudaStream_t s) const {
    if (p) a.free(a.ctx, p, bytes, (void*)s);
}
}  // namespace mc

struct mc_db {
    mc::Mem mem;
    cudaStream_t stream = nullptr;
    mc::SketchParams sp{};
    uint32_t cap = 0;
    uint64_t hbm_budget = 0;
    // taxonomy
    uint32_t n_taxa = 0;
    std::vector<uint32_t> parent;  // host copy, for mc_db_save
    DevBuf depth, lineage;
    uint32_t lin_stride = 0, max_depth = 0;
    // targets
    uint32_t n_targets = 0;
    DevBuf taxon;  // u32 per target
    DevBuf wbase;  // u32 global window base per target, n_targets+1 entries
    uint64_t n_windows = 0;
    uint64_t max_target_windows = 0;  // most windows of one target
    // additions not yet finalized
    DevBuf pending;  // u64 pairs
    uint64_t pending_n = 0, pending_real = 0;
    bool pending_sorted = false;  // pending holds pending_real sorted pairs (mc_db_feature_counts)
    // published condensed layout: locations in the loc_jbits encoding
    // (mc::loc_bytes), packed feature-table words in format fmt
    DevBuf locs, table;
    uint64_t n_kept = 0, n_keys = 0, table_len = 0, overflow_keys = 0, n_pairs = 0;
    mc::TableFmt fmt{1, 1};
    uint32_t max_probe = 0, loc_jbits = 0;
    bool dirty = false, has_table = false;
    // a finalize failed after its sort had consumed the pending pairs: the
    // last published layout still serves classification, but nothing can
    // be added or finalized any more
    bool failed = false;
    uint64_t epoch = 0;  // finalizes so far (plans re-capture when it changes)
    cudaEvent_t ready = nullptr;
    DevBuf status;  // u32 device status word
    mc::Tuning tuning = mc::DEFAULT_TUNING;
    // streams that classified against this database, each with an event
    // recorded after its last classify launches: buffers those launches may
    // read are freed only after the database stream has waited on them
    struct StreamUse {
        cudaStream_t s;
        cudaEvent_t ev;
    };
    mutable std::mutex use_mu;
    mutable std::vector<StreamUse> uses;
};

namespace {

void release(mc_db* db, DevBuf& b) {
    if (b.p) db->mem.free(b.p, b.bytes, db->stream);
    b = DevBuf();
}

bool grab(mc_db* db, DevBuf& b, size_t bytes) {
    b.p = bytes ? db->mem.alloc(bytes, db->stream) : nullptr;
    b.bytes = bytes;
    return bytes == 0 || b.p != nullptr;
}

// Records that classify work was enqueued on `s`.
cudaError_t note_use(const mc_db* db, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(db->use_mu);
    for (auto& u : db->uses)
        if (u.s == s) return cudaEventRecord(u.ev, s);
    mc_db::StreamUse u{s, nullptr};
    cudaError_t e = cudaEventCreateWithFlags(&u.ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    db->uses.push_back(u);
    return cudaEventRecord(u.ev, s);
}

// Makes the database stream wait for every classify enqueued so far.
void wait_uses(mc_db* db) {
    std::lock_guard<std::mutex> lock(db->use_mu);
    for (auto& u : db->uses) cudaStreamWaitEvent(db->stream, u.ev, 0);
}

// Releases a buffer that classify launches may still read.
void retire(mc_db* db, DevBuf& b) {
    if (!b.p) return;
    wait_uses(db);
    release(db, b);
}

uint64_t held_bytes(const mc_db* db) {
    return db->depth.bytes + db->lineage.bytes + db->taxon.bytes + db->wbase.bytes + db->pending.bytes +
           db->locs.bytes + db->table.bytes + db->status.bytes;
}

bool within_budget(const mc_db* db, uint64_t extra) {
    return db->hbm_budget == 0 || held_bytes(db) + extra <= db->hbm_budget;
}

// Grows b to hold at least `need` bytes, keeping the first `keep` bytes.
int grow(mc_db* db, DevBuf& b, size_t need, size_t keep, const char* what) {
    if (b.bytes >= need) return MC_OK;
    size_t nb = std::max(need, b.bytes + b.bytes / 2);
    if (!within_budget(db, nb)) return fail(MC_ERR_OOM, "%s: hbm_budget exceeded", what);
    DevBuf n;
    if (!grab(db, n, nb)) return fail(MC_ERR_OOM, "%s: cannot allocate %zu bytes", what, nb);
    if (keep) MC_CU(cudaMemcpyAsync(n.p, b.p, keep, cudaMemcpyDeviceToDevice, db->stream));
    retire(db, b);
    b = n;
    return MC_OK;
}

int check_params(const mc_db_params* p) {
    if (!p) return fail(MC_ERR_ARG, "params is NULL");
    if (p->k < 1 || p->k > MC_MAX_K) return fail(MC_ERR_ARG, "k must be in 1..%d", MC_MAX_K);
    if (p->sketch_size < 1 || p->sketch_size > MC_MAX_SKETCH)
        return fail(MC_ERR_ARG, "sketch_size must be in 1..%d", MC_MAX_SKETCH);
    if (p->window_len < p->k || p->window_len > 512) return fail(MC_ERR_ARG, "window_len must be in k..512");
    if (p->window_len - p->k + 1 > MC_MAX_WINDOW_KMERS) return fail(MC_ERR_ARG, "window has too many k-mers");
    if (p->window_stride < 1 || p->window_stride > p->window_len - p->k + 1)
        return fail(MC_ERR_ARG, "window_stride must be in 1..window_len-k+1");
    if (p->bucket_cap < 1 || p->bucket_cap > 65535) return fail(MC_ERR_ARG, "bucket_cap must be in 1..65535");
    if (p->reserved != 0) return fail(MC_ERR_ARG, "reserved must be 0");
    return MC_OK;
}

mc::SketchParams sketch_params(const mc_db_params* p) {
    return mc::SketchParams{p->k, p->sketch_size, p->window_len, p->window_stride};
}

int check_cls(const mc_classify_params* p) {
    if (!p) return fail(MC_ERR_ARG, "classify params is NULL");
    if (p->max_candidates < 1 || p->max_candidates > MC_MAX_CANDIDATES)
        return fail(MC_ERR_ARG, "max_candidates must be in 1..%d", MC_MAX_CANDIDATES);
    if (p->lca_band_pct > 100) return fail(MC_ERR_ARG, "lca_band_pct must be in 0..100");
    if (p->max_insert > MC_MAX_INSERT) return fail(MC_ERR_ARG, "max_insert must be <= %d", MC_MAX_INSERT);
    return MC_OK;
}

// Kernel view of a finalized database.
mc::ClassifyDb db_view(const mc_db* db) {
    mc::ClassifyDb cdb;
    cdb.table = (const uint64_t*)db->table.p;
    cdb.fmt = db->fmt;
    cdb.max_probe = db->max_probe;
    cdb.locs = db->locs.p;
    cdb.taxon_of_target = (const uint32_t*)db->taxon.p;
    cdb.n_targets = db->n_targets;
    cdb.lineage = (const uint32_t*)db->lineage.p;
    cdb.depth = (const uint32_t*)db->depth.p;
    cdb.lin_stride = db->lin_stride;
    cdb.n_taxa = db->n_taxa;
    cdb.sp = db->sp;
    cdb.jbits = db->loc_jbits;
    return cdb;
}

}  // namespace

extern "C" {

int mc_version(void) { return MC_API_VERSION; }

uint64_t mc_kernel_launches(void) { return g_launches.load(); }

int mc_trace_enable(int on) {
    g_trace_on.store(on ? 1 : 0);
    return MC_OK;
}

int mc_trace_report(char* buf, size_t len, int reset) {
    std::lock_guard<std::mutex> lock(g_trace_mu);
    for (TraceRec& r : g_trace_pending) {
        float ms = 0;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            auto it = std::find_if(g_trace_acc.begin(), g_trace_acc.end(),
                                   [&](const std::pair<std::string, TraceAcc>& x) { return x.first == r.name; });
            if (it == g_trace_acc.end()) {
                g_trace_acc.push_back({r.name, TraceAcc()});
                it = g_trace_acc.end() - 1;
            }
            it->second.n += 1;
            it->second.ms += ms;
        }
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    cudaGetLastError();
    g_trace_pending.clear();
    std::string out;
    char line[256];
    for (auto& x : g_trace_acc) {
        snprintf(line, sizeof line, "%s %llu %.6f\n", x.first.c_str(), (unsigned long long)x.second.n, x.second.ms);
        out += line;
    }
    if (buf && len) {
        size_t n = std::min(len - 1, out.size());
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    if (reset) g_trace_acc.clear();
    return (int)out.size();
}

const char* mc_last_error_string(void) { return g_err; }

const char* mc_status_string(int s) {
    switch (s) {
        case MC_OK: return "MC_OK";
        case MC_ERR_ARG: return "MC_ERR_ARG";
        case MC_ERR_STATE: return "MC_ERR_STATE";
        case MC_ERR_OOM: return "MC_ERR_OOM";
        case MC_ERR_TABLE_FULL: return "MC_ERR_TABLE_FULL";
        case MC_ERR_TIMEOUT: return "MC_ERR_TIMEOUT";
        case MC_ERR_CUDA: return "MC_ERR_CUDA";
        case MC_ERR_CAPACITY: return "MC_ERR_CAPACITY";
        default: return "unknown";
    }
}

int mc_set_allocator(const mc_allocator* a) {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    if (a && (!a->alloc || !a->free)) return fail(MC_ERR_ARG, "allocator needs alloc and free");
    g_alloc = a ? *a : mc_allocator{default_alloc, default_free, nullptr};
    return MC_OK;
}

int mc_db_create(const mc_db_params* params, uint32_t n_taxa, const uint32_t* parent, void* stream, mc_db** out) {
    g_err[0] = 0;
    if (!out) return fail(MC_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = check_params(params);
    if (rc) return rc;
    if (n_taxa < 1) return fail(MC_ERR_ARG, "n_taxa must be >= 1");
    if (!parent) return fail(MC_ERR_ARG, "parent is NULL");
    for (uint32_t i = 0; i < n_taxa; ++i)
        if (parent[i] >= n_taxa) return fail(MC_ERR_ARG, "parent[%u] = %u is out of range", i, parent[i]);
    mc_db* db = new mc_db();
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        db->mem.a = g_alloc;
        if (g_alloc.alloc == default_alloc) configure_default_pool();
    }
    db->stream = (cudaStream_t)stream;
    db->sp = sketch_params(params);
    db->cap = params->bucket_cap;
    db->hbm_budget = params->hbm_budget;
    db->n_taxa = n_taxa;
    db->parent.assign(parent, parent + n_taxa);
    auto bail = [&](int code) {
        mc_db_free(db);
        return code;
    };
    if (cudaEventCreateWithFlags(&db->ready, cudaEventDisableTiming) != cudaSuccess)
        return bail(cuda_fail(cudaGetLastError(), "cudaEventCreate"));
    DevBuf d_parent, flags;
    if (!grab(db, d_parent, (size_t)n_taxa * 4) || !grab(db, db->depth, (size_t)n_taxa * 4) ||
        !grab(db, flags, 8) || !grab(db, db->status, 4))
        return bail(fail(MC_ERR_OOM, "mc_db_create: allocation failed"));
    auto free_tmp = [&]() {
        release(db, d_parent);
        release(db, flags);
    };
    uint32_t host_flags[2] = {0, 0};
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_parent.p, parent, (size_t)n_taxa * 4, cudaMemcpyHostToDevice, db->stream)) ||
        (e = cudaMemsetAsync(flags.p, 0, 8, db->stream)) || (e = cudaMemsetAsync(db->status.p, 0, 4, db->stream)) ||
        (e = mc::taxonomy_depths((uint32_t*)d_parent.p, n_taxa, (uint32_t*)db->depth.p, (uint32_t*)flags.p,
                                 (uint32_t*)flags.p + 1, db->stream)) ||
        (e = cudaMemcpyAsync(host_flags, flags.p, 8, cudaMemcpyDeviceToHost, db->stream)) ||
        (e = cudaStreamSynchronize(db->stream))) {
        free_tmp();
        return bail(cuda_fail(e, "mc_db_create taxonomy"));
    }
    if (host_flags[1]) {
        free_tmp();
        return bail(fail(MC_ERR_ARG, "parent array has a cycle"));
    }
    db->max_depth = host_flags[0];
    db->lin_stride = db->max_depth + 1;
    if (!grab(db, db->lineage, (size_t)n_taxa * db->lin_stride * 4)) {
        free_tmp();
        return bail(fail(MC_ERR_OOM, "mc_db_create: lineage allocation failed"));
    }
    if ((e = mc::taxonomy_lineage((uint32_t*)d_parent.p, n_taxa, (uint32_t*)db->depth.p, (uint32_t*)db->lineage.p,
                                  db->lin_stride, db->stream)) ||
        (e = cudaStreamSynchronize(db->stream))) {
        free_tmp();
        return bail(cuda_fail(e, "mc_db_create lineage"));
    }
    free_tmp();
    // window base of target 0
    if (!grab(db, db->wbase, 4 * 1024)) return bail(fail(MC_ERR_OOM, "mc_db_create: allocation failed"));
    if ((e = cudaMemsetAsync(db->wbase.p, 0, 4, db->stream)) || (e = cudaStreamSynchronize(db->stream)))
        return bail(cuda_fail(e, "mc_db_create"));
    *out = db;
    return MC_OK;
}

int mc_db_add_targets(mc_db* db, uint32_t n_targets, const char* seq, const uint64_t* offs, const uint32_t* taxon,
                      uint32_t* first_target_id) {
    g_err[0] = 0;
    if (!db) return fail(MC_ERR_ARG, "db is NULL");
    if (db->failed) return fail(MC_ERR_STATE, "the database cannot grow after a failed mc_db_finalize");
    if (first_target_id) *first_target_id = db->n_targets;
    if (n_targets == 0) return MC_OK;
    if (!seq || !offs || !taxon) return fail(MC_ERR_ARG, "seq, offs and taxon must not be NULL");
    if ((uint64_t)db->n_targets + n_targets >= 0xFFFFFFFFull) return fail(MC_ERR_CAPACITY, "too many targets");
    for (uint32_t i = 0; i < n_targets; ++i)
        if (taxon[i] >= db->n_taxa && taxon[i] != MC_NO_TAXON)
            return fail(MC_ERR_ARG, "taxon[%u] = %u is out of range", i, taxon[i]);
    cudaStream_t s = db->stream;
    mc::Tmp<uint64_t> win_offs(db->mem, (size_t)n_targets + 1, s);
    mc::Tmp<unsigned long long> ctr(db->mem, 2, s);
    if (!win_offs.ok() || !ctr.ok()) return fail(MC_ERR_OOM, "mc_db_add_targets: allocation failed");
    MC_CU(cudaMemsetAsync(ctr.ptr, 0, 16, s));
    MC_CU(mc::window_offsets(db->mem, db->sp, n_targets, offs, win_offs.ptr, (uint32_t*)ctr.ptr, s));
    uint64_t nw = 0;
    unsigned long long bad = 0;
    MC_CU(cudaMemcpyAsync(&nw, win_offs.ptr + n_targets, 8, cudaMemcpyDeviceToHost, s));
    MC_CU(cudaMemcpyAsync(&bad, ctr.ptr, 8, cudaMemcpyDeviceToHost, s));
    MC_CU(cudaStreamSynchronize(s));
    if (bad) return fail(MC_ERR_ARG, "offs must be non-decreasing");
    if (db->n_windows + nw >= 0xFFFFFFFFull) return fail(MC_ERR_CAPACITY, "more than 2^32-2 windows");
    int rc;
    const uint32_t t0 = db->n_targets;
    if ((rc = grow(db, db->taxon, (size_t)(t0 + n_targets) * 4, (size_t)t0 * 4, "taxon"))) return rc;
    if ((rc = grow(db, db->wbase, (size_t)(t0 + n_targets + 1) * 4, (size_t)(t0 + 1) * 4, "wbase"))) return rc;
    const uint64_t npairs = nw * db->sp.s;
    if ((rc = grow(db, db->pending, (db->pending_n + npairs) * 8, db->pending_n * 8, "pending pairs"))) return rc;
    MC_CU(cudaMemcpyAsync((uint32_t*)db->taxon.p + t0, taxon, (size_t)n_targets * 4, cudaMemcpyHostToDevice, s));
    // global window bases of the new targets: n_windows + win_offs[i]
    {
        std::vector<uint64_t> h(n_targets + 1);
        MC_CU(cudaMemcpyAsync(h.data(), win_offs.ptr, h.size() * 8, cudaMemcpyDeviceToHost, s));
        MC_CU(cudaStreamSynchronize(s));
        std::vector<uint32_t> wb(n_targets + 1);
        for (uint32_t i = 0; i <= n_targets; ++i) wb[i] = (uint32_t)(db->n_windows + h[i]);
        for (uint32_t i = 0; i < n_targets; ++i) db->max_target_windows = std::max(db->max_target_windows, h[i + 1] - h[i]);
        MC_CU(cudaMemcpyAsync((uint32_t*)db->wbase.p + t0, wb.data(), wb.size() * 4, cudaMemcpyHostToDevice, s));
        MC_CU(mc::emit_pairs(db->sp, n_targets, (const uint8_t*)seq, offs, win_offs.ptr, nw, (uint32_t)db->n_windows,
                             (uint64_t*)db->pending.p + db->pending_n, ctr.ptr + 1, s));
        unsigned long long real = 0;
        MC_CU(cudaMemcpyAsync(&real, ctr.ptr + 1, 8, cudaMemcpyDeviceToHost, s));
        MC_CU(cudaStreamSynchronize(s));
        db->pending_n += npairs;
        db->pending_real += real;
        db->pending_sorted = false;
    }
    db->n_windows += nw;
    db->n_targets += n_targets;
    db->dirty = true;
    return MC_OK;
}

}  // extern "C"

namespace {
// mc_db_finalize with an optional prior (sharded builds): n_lists lists of
// earlier shards' feature counts.
int finalize_impl(mc_db* db, uint32_t n_lists, const uint32_t* const* keys, const uint32_t* const* counts,
                  const uint64_t* list_n) {
    g_err[0] = 0;
    if (!db) return fail(MC_ERR_ARG, "db is NULL");
    if (db->failed) return fail(MC_ERR_STATE, "an earlier mc_db_finalize failed after consuming the added targets");
    if (!db->dirty && db->has_table) return MC_OK;
    cudaStream_t s = db->stream;
    const uint64_t n_old = db->n_kept;
    // 1. the new pairs are sorted (unless mc_db_feature_counts did it): the
    // sort allocates its scratch before it touches the pairs, so a refused
    // allocation leaves them as they were and the call can be repeated
    if (!db->pending_sorted && db->pending_n) {
        DevBuf b;
        if (!grab(db, b, db->pending_n * 8)) return fail(MC_ERR_OOM, "finalize: allocation failed");
        cudaError_t e = mc::sort_pairs(db->mem, (uint64_t*)db->pending.p, (uint64_t*)b.p, db->pending_n,
                                       db->pending_real, s);
        release(db, b);
        if (e != cudaSuccess) {
            if (e != cudaErrorMemoryAllocation) db->failed = true;
            return cuda_fail(e, "finalize: sort");
        }
        db->pending_n = db->pending_real;  // the first pending_real pairs are sorted, the rest is stale
        db->pending_sorted = true;
    }
    const uint64_t n_new = db->pending_real;
    const uint64_t n_real = n_old + n_new;
    // 2. live extension (Section 4.1: new targets get the next ids, so every
    // new location is larger than the stored ones): the stored pairs, in
    // layout order, are already sorted; merging them with the new pairs
    // gives the sorted pairs of the whole database without sorting the
    // stored ones again.  Without a stored layout the new pairs are it.
    DevBuf a;
    const bool a_is_pending = n_old == 0;
    if (a_is_pending) {
        a = db->pending;
    } else {
        DevBuf old;
        if (!within_budget(db, (n_old + n_real) * 8)) return fail(MC_ERR_OOM, "finalize: hbm_budget exceeded");
        if (!grab(db, old, n_old * 8) || !grab(db, a, n_real * 8)) {
            release(db, old);
            release(db, a);
            return fail(MC_ERR_OOM, "finalize: allocation failed");
        }
        cudaError_t e = mc::reconstruct_pairs((const uint64_t*)db->table.p, db->table_len, db->fmt, db->locs.p,
                                              db->loc_jbits, (const uint32_t*)db->wbase.p, (uint64_t*)old.p, s);
        if (e == cudaSuccess)
            e = mc::merge_sorted_pairs((const uint64_t*)old.p, n_old, (const uint64_t*)db->pending.p, n_new,
                                       (uint64_t*)a.p, s);
        release(db, old);
        if (e != cudaSuccess) {
            release(db, a);
            return cuda_fail(e, "finalize: merge of the stored pairs");
        }
    }
    auto release_tmp = [&]() {
        if (!a_is_pending) release(db, a);
    };
    uint64_t prior_over = 0;
    if (n_lists) {
        cudaError_t e = mc::apply_prior(db->mem, (uint64_t*)a.p, n_real, db->cap, n_lists, keys, counts, list_n,
                                        &prior_over, s);
        if (e != cudaSuccess) {
            release_tmp();
            db->failed = true;
            return cuda_fail(e, "finalize: prior counts");
        }
    }
    mc::FinalizeOut fo;
    const uint32_t jbits = mc::compact_key_bits(db->n_targets, db->max_target_windows);
    cudaError_t e = mc::finalize_pairs(db->mem, (const uint64_t*)a.p, n_real, db->cap, (const uint32_t*)db->wbase.p,
                                       db->n_targets, jbits, &fo, s);
    release_tmp();
    if (e != cudaSuccess) {
        db->failed = true;
        return cuda_fail(e, "finalize: layout");
    }
    if (fo.table_full) {
        db->failed = true;
        return fail(MC_ERR_TABLE_FULL, "finalize: %llu features and %llu locations fit no feature-table format",
                    (unsigned long long)fo.n_keys, (unsigned long long)fo.n_kept);
    }
    release(db, db->pending);
    retire(db, db->locs);
    retire(db, db->table);
    db->locs = DevBuf{fo.locs, fo.n_kept * mc::loc_bytes(jbits)};
    db->table = DevBuf{fo.table, fo.table_bytes};
    db->loc_jbits = jbits;
    db->n_pairs += db->pending_real;
    db->pending_n = db->pending_real = 0;
    db->pending_sorted = false;
    db->n_kept = fo.n_kept;
    db->n_keys = fo.n_keys;
    db->table_len = fo.table_len;
    db->fmt = fo.fmt;
    db->max_probe = fo.max_probe;
    db->overflow_keys = fo.overflow_keys + prior_over;
    db->dirty = false;
    db->has_table = true;
    ++db->epoch;
    MC_CU(cudaEventRecord(db->ready, s));
    MC_CU(cudaStreamSynchronize(s));
    return MC_OK;
}
}  // namespace

extern "C" {

int mc_db_finalize(mc_db* db) { return finalize_impl(db, 0, nullptr, nullptr, nullptr); }

int mc_db_feature_counts(mc_db* db, uint64_t max_keys, uint32_t* keys, uint32_t* counts, uint64_t* n_keys) {
    g_err[0] = 0;
    if (!db || !n_keys) return fail(MC_ERR_ARG, "NULL argument");
    *n_keys = 0;
    if (db->failed) return fail(MC_ERR_STATE, "an earlier mc_db_finalize failed");
    if (db->has_table) return fail(MC_ERR_STATE, "mc_db_feature_counts: the database was finalized already");
    cudaStream_t s = db->stream;
    if (!db->pending_sorted && db->pending_n) {
        DevBuf b;
        if (!grab(db, b, db->pending_n * 8)) return fail(MC_ERR_OOM, "mc_db_feature_counts: allocation failed");
        cudaError_t e = mc::sort_pairs(db->mem, (uint64_t*)db->pending.p, (uint64_t*)b.p, db->pending_n,
                                       db->pending_real, s);
        release(db, b);
        if (e != cudaSuccess) {
            if (e != cudaErrorMemoryAllocation) db->failed = true;
            return cuda_fail(e, "mc_db_feature_counts: sort");
        }
        // the first pending_real pairs are sorted, the rest is stale
        db->pending_n = db->pending_real;
        db->pending_sorted = true;
    }
    uint64_t n = 0;
    MC_CU(mc::feature_counts(db->mem, (const uint64_t*)db->pending.p, db->pending_real, db->cap, max_keys, keys,
                             counts, &n, s));
    *n_keys = n;
    if (n > max_keys) return fail(MC_ERR_CAPACITY, "mc_db_feature_counts: %llu features", (unsigned long long)n);
    return MC_OK;
}

int mc_db_finalize_after(mc_db* db, uint32_t n_lists, const uint32_t* const* keys, const uint32_t* const* counts,
                         const uint64_t* n_keys) {
    g_err[0] = 0;
    if (n_lists && (!keys || !counts || !n_keys)) return fail(MC_ERR_ARG, "NULL prior list arrays");
    for (uint32_t l = 0; l < n_lists; ++l)
        if (n_keys[l] && (!keys[l] || !counts[l])) return fail(MC_ERR_ARG, "prior list %u has NULL arrays", l);
    return finalize_impl(db, n_lists, keys, counts, n_keys);
}

static int classify_impl(const mc_db* db, const mc_classify_params* params, uint32_t n_seq, const char* seq,
                         const uint64_t* offs, uint32_t n_queries, const uint32_t* qoffs, uint32_t* label,
                         uint32_t* hits, uint32_t* top_target, uint32_t* cands, uint64_t* counters, void* stream) {
    g_err[0] = 0;
    if (!db) return fail(MC_ERR_ARG, "db is NULL");
    int rc = check_cls(params);
    if (rc) return rc;
    if (!db->has_table) return fail(MC_ERR_STATE, "mc_classify before mc_db_finalize");
    if (n_queries == 0) return MC_OK;
    if (!seq || !offs || !qoffs || !label || !hits) return fail(MC_ERR_ARG, "NULL input or output pointer");
    (void)n_seq;
    cudaStream_t s = (cudaStream_t)stream;
    MC_CU(cudaStreamWaitEvent(s, db->ready, 0));
    const mc::ClassifyDb cdb = db_view(db);
    mc::ClassifyQuery q;
    q.seq = (const uint8_t*)seq;
    q.offs = offs;
    q.qoffs = qoffs;
    q.n_q = n_queries;
    q.m = params->max_candidates;
    q.hits_min = params->hits_min;
    q.band = params->lca_band_pct;
    q.max_insert = params->max_insert;
    q.label = label;
    q.hits = hits;
    q.top_target = top_target;
    q.cands = cands;
    q.counters = (unsigned long long*)counters;
    q.status = (uint32_t*)db->status.p;
    q.batches = nullptr;
    q.bhdr = nullptr;
    MC_CU(mc::classify_launch(db->mem, cdb, q, db->tuning, s));
    MC_CU(note_use(db, s));
    return MC_OK;
}

}  // extern "C"

namespace mc {
int report_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

int classify_prepare(const mc_db* db, const mc_classify_params* params, const char* seq, const uint64_t* offs,
                     uint32_t n_queries, const uint32_t* qoffs, uint32_t* label, uint32_t* hits,
                     uint32_t* top_target, cudaStream_t stream, ClassifyDb* cdb, ClassifyQuery* q) {
    g_err[0] = 0;
    if (!db) return fail(MC_ERR_ARG, "db is NULL");
    int rc = check_cls(params);
    if (rc) return rc;
    if (!db->has_table) return fail(MC_ERR_STATE, "classify before mc_db_finalize");
    if (n_queries && (!seq || !offs || !qoffs || !label || !hits))
        return fail(MC_ERR_ARG, "NULL input or output pointer");
    MC_CU(cudaStreamWaitEvent(stream, db->ready, 0));
    *cdb = db_view(db);
    q->seq = (const uint8_t*)seq;
    q->offs = offs;
    q->qoffs = qoffs;
    q->n_q = n_queries;
    q->m = params->max_candidates;
    q->hits_min = params->hits_min;
    q->band = params->lca_band_pct;
    q->max_insert = params->max_insert;
    q->label = label;
    q->hits = hits;
    q->top_target = top_target;
    q->cands = nullptr;
    q->counters = nullptr;
    q->status = (uint32_t*)db->status.p;
    q->batches = nullptr;
    q->bhdr = nullptr;
    return MC_OK;
}

Tuning db_tuning(const mc_db* db) { return db->tuning; }

int classify_done(const mc_db* db, cudaStream_t stream) {
    cudaError_t e = note_use(db, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return report_error(MC_ERR_CUDA, "classify: %s", cudaGetErrorString(e));
    }
    return MC_OK;
}
}  // namespace mc

extern "C" {

int mc_classify(const mc_db* db, const mc_classify_params* params, uint32_t n_seq, const char* seq,
                const uint64_t* offs, uint32_t n_queries, const uint32_t* qoffs, uint32_t* label, uint32_t* hits,
                uint32_t* top_target, void* stream) {
    return classify_impl(db, params, n_seq, seq, offs, n_queries, qoffs, label, hits, top_target, nullptr, nullptr,
                         stream);
}

int mc_classify_debug(const mc_db* db, const mc_classify_params* params, uint32_t n_seq, const char* seq,
                      const uint64_t* offs, uint32_t n_queries, const uint32_t* qoffs, uint32_t* label,
                      uint32_t* hits, uint32_t* top_target, uint32_t* cands, uint64_t* counters, void* stream) {
    return classify_impl(db, params, n_seq, seq, offs, n_queries, qoffs, label, hits, top_target, cands, counters,
                         stream);
}

int mc_debug_stall_next_sort(uint64_t limit_ns) {
    g_err[0] = 0;
    if (limit_ns < 1000000ull || limit_ns > 2000000000ull)
        return fail(MC_ERR_ARG, "mc_debug_stall_next_sort: limit must be in 1e6..2e9 ns");
    mc::arm_sort_stall(limit_ns);
    return MC_OK;
}

int mc_merge_candidates(const mc_db* db, const mc_classify_params* params, uint32_t n_queries, uint32_t n_lists,
                        const uint32_t* const* cands, const uint32_t* target_base, const uint32_t* taxon_of_target,
                        uint32_t n_targets, uint32_t* label, uint32_t* hits, uint32_t* top_target,
                        uint32_t* cands_out, void* stream) {
    g_err[0] = 0;
    if (!db) return fail(MC_ERR_ARG, "db is NULL");
    int rc = check_cls(params);
    if (rc) return rc;
    if (n_queries == 0) return MC_OK;
    if (!label || !hits || (n_lists && (!cands || !target_base)) || (n_targets && !taxon_of_target))
        return fail(MC_ERR_ARG, "NULL argument");
    std::vector<mc::MergeList> lists(n_lists);
    for (uint32_t l = 0; l < n_lists; ++l) {
        if (!cands[l]) return fail(MC_ERR_ARG, "candidate list %u is NULL", l);
        lists[l] = mc::MergeList{cands[l], target_base[l]};
    }
    MC_CU(mc::merge_candidates(db->mem, db_view(db), taxon_of_target, n_targets, lists.data(), n_lists, n_queries,
                               params->max_candidates, params->hits_min, params->lca_band_pct, label, hits, top_target,
                               cands_out, (cudaStream_t)stream));
    return MC_OK;
}

int mc_classify_status(const mc_db* db, void* stream) {
    g_err[0] = 0;
    if (!db) return fail(MC_ERR_ARG, "db is NULL");
    MC_CU(cudaStreamSynchronize((cudaStream_t)stream));
    uint32_t st = 0;
    MC_CU(cudaMemcpy(&st, db->status.p, 4, cudaMemcpyDeviceToHost));
    MC_CU(cudaMemset(db->status.p, 0, 4));
    if (st == mc::DEV_ERR_CAPACITY)
        return fail(MC_ERR_CAPACITY, "a query exceeded the per-query window or histogram capacity");
    if (st) return fail(MC_ERR_ARG, "device reported status %u", st);
    return MC_OK;
}

void mc_db_free(mc_db* db) {
    if (!db) return;
    cudaStreamSynchronize(db->stream);
    release(db, db->depth);
    release(db, db->lineage);
    release(db, db->taxon);
    release(db, db->wbase);
    release(db, db->pending);
    release(db, db->locs);
    release(db, db->table);
    release(db, db->status);
    cudaStreamSynchronize(db->stream);
    if (db->ready) cudaEventDestroy(db->ready);
    cudaGetLastError();
    delete db;
}

namespace {
const char MAGIC[8] = {'M', 'C', 'G', 'B', '3', 'D', 'B', '1'};
const uint32_t FILE_VERSION = 2;

// Format 2: 8-byte feature-table words (log_t, cbits) and locations in the
// loc_jbits encoding.
struct FileHeader {
    char magic[8];
    uint32_t version, k, s, w, stride, cap, n_taxa, n_targets, log_t, max_probe, cbits, loc_jbits;
    uint64_t n_windows, n_pairs, n_keys, n_kept, table_len, overflow_keys;
};

// Device <-> file through a host staging buffer.
int write_device(FILE* f, const void* dev, size_t bytes, cudaStream_t s, std::vector<char>& stage) {
    const size_t chunk = stage.size();
    for (size_t off = 0; off < bytes; off += chunk) {
        const size_t n = std::min(chunk, bytes - off);
        MC_CU(cudaMemcpyAsync(stage.data(), (const char*)dev + off, n, cudaMemcpyDeviceToHost, s));
        MC_CU(cudaStreamSynchronize(s));
        if (fwrite(stage.data(), 1, n, f) != n) return fail(MC_ERR_ARG, "mc_db_save: write failed");
    }
    return MC_OK;
}

int read_device(FILE* f, void* dev, size_t bytes, cudaStream_t s, std::vector<char>& stage) {
    const size_t chunk = stage.size();
    for (size_t off = 0; off < bytes; off += chunk) {
        const size_t n = std::min(chunk, bytes - off);
        if (fread(stage.data(), 1, n, f) != n) return fail(MC_ERR_ARG, "mc_db_load: file is truncated");
        MC_CU(cudaMemcpyAsync((char*)dev + off, stage.data(), n, cudaMemcpyHostToDevice, s));
        MC_CU(cudaStreamSynchronize(s));
    }
    return MC_OK;
}
}  // namespace

int mc_db_save(const mc_db* db, const char* path) {
    g_err[0] = 0;
    if (!db || !path) return fail(MC_ERR_ARG, "NULL argument");
    if (!db->has_table || db->dirty) return fail(MC_ERR_STATE, "mc_db_save: finalize the database first");
    FILE* f = fopen(path, "wb");
    if (!f) return fail(MC_ERR_ARG, "mc_db_save: cannot open %s", path);
    FileHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, MAGIC, 8);
    h.version = FILE_VERSION;
    h.k = db->sp.k;
    h.s = db->sp.s;
    h.w = db->sp.w;
    h.stride = db->sp.stride;
    h.cap = db->cap;
    h.n_taxa = db->n_taxa;
    h.n_targets = db->n_targets;
    h.log_t = db->fmt.log_t;
    h.cbits = db->fmt.cbits;
    h.loc_jbits = db->loc_jbits;
    h.max_probe = db->max_probe;
    h.n_windows = db->n_windows;
    h.n_pairs = db->n_pairs;
    h.n_keys = db->n_keys;
    h.n_kept = db->n_kept;
    h.table_len = db->table_len;
    h.overflow_keys = db->overflow_keys;
    std::vector<char> stage(64u << 20);
    int rc = MC_OK;
    if (fwrite(&h, sizeof h, 1, f) != 1 || fwrite(db->parent.data(), 4, db->n_taxa, f) != db->n_taxa)
        rc = fail(MC_ERR_ARG, "mc_db_save: write failed");
    if (!rc) rc = write_device(f, db->taxon.p, (size_t)db->n_targets * 4, db->stream, stage);
    if (!rc) rc = write_device(f, db->wbase.p, ((size_t)db->n_targets + 1) * 4, db->stream, stage);
    if (!rc) rc = write_device(f, db->locs.p, db->n_kept * mc::loc_bytes(db->loc_jbits), db->stream, stage);
    if (!rc) rc = write_device(f, db->table.p, db->table_len * sizeof(uint64_t), db->stream, stage);
    if (fclose(f) != 0 && !rc) rc = fail(MC_ERR_ARG, "mc_db_save: close failed");
    return rc;
}

int mc_db_load(const char* path, void* stream, mc_db** out) {
    g_err[0] = 0;
    if (!path || !out) return fail(MC_ERR_ARG, "NULL argument");
    *out = nullptr;
    FILE* f = fopen(path, "rb");
    if (!f) return fail(MC_ERR_ARG, "mc_db_load: cannot open %s", path);
    FileHeader h;
    if (fread(&h, sizeof h, 1, f) != 1 || std::memcmp(h.magic, MAGIC, 8) != 0) {
        fclose(f);
        return fail(MC_ERR_ARG, "mc_db_load: %s is not a database file", path);
    }
    if (h.version != FILE_VERSION) {
        fclose(f);
        return fail(MC_ERR_ARG, "mc_db_load: format version %u, expected %u", h.version, FILE_VERSION);
    }
    std::vector<uint32_t> parent(h.n_taxa);
    if (h.n_taxa == 0 || fread(parent.data(), 4, h.n_taxa, f) != h.n_taxa) {
        fclose(f);
        return fail(MC_ERR_ARG, "mc_db_load: file is truncated");
    }
    mc_db_params p;
    std::memset(&p, 0, sizeof p);
    p.k = h.k;
    p.sketch_size = h.s;
    p.window_len = h.w;
    p.window_stride = h.stride;
    p.bucket_cap = h.cap;
    mc_db* db = nullptr;
    int rc = mc_db_create(&p, h.n_taxa, parent.data(), stream, &db);
    if (rc) {
        fclose(f);
        return rc;
    }
    std::vector<char> stage(64u << 20);
    if (h.log_t < 1 || h.log_t > 32 || h.cbits != mc::count_bits(h.cap) || h.loc_jbits > 31 || h.max_probe > mc::TAB_MAX_DISP) {
        fclose(f);
        mc_db_free(db);
        return fail(MC_ERR_ARG, "mc_db_load: %s has an invalid table format", path);
    }
    const size_t loc_b = mc::loc_bytes(h.loc_jbits);
    if (!grab(db, db->taxon, std::max<size_t>((size_t)h.n_targets * 4, 4)) ||
        !grab(db, db->locs, h.n_kept * loc_b) || !grab(db, db->table, h.table_len * sizeof(uint64_t))) {
        fclose(f);
        mc_db_free(db);
        return fail(MC_ERR_OOM, "mc_db_load: allocation failed");
    }
    release(db, db->wbase);
    if (!grab(db, db->wbase, ((size_t)h.n_targets + 1) * 4)) {
        fclose(f);
        mc_db_free(db);
        return fail(MC_ERR_OOM, "mc_db_load: allocation failed");
    }
    rc = read_device(f, db->taxon.p, (size_t)h.n_targets * 4, db->stream, stage);
    if (!rc) rc = read_device(f, db->wbase.p, ((size_t)h.n_targets + 1) * 4, db->stream, stage);
    if (!rc) rc = read_device(f, db->locs.p, h.n_kept * loc_b, db->stream, stage);
    if (!rc) rc = read_device(f, db->table.p, h.table_len * sizeof(uint64_t), db->stream, stage);
    fclose(f);
    if (rc) {
        mc_db_free(db);
        return rc;
    }
    db->n_targets = h.n_targets;
    db->n_windows = h.n_windows;
    db->n_pairs = h.n_pairs;
    db->n_keys = h.n_keys;
    db->n_kept = h.n_kept;
    db->table_len = h.table_len;
    db->fmt = mc::TableFmt{h.log_t, h.cbits};
    db->loc_jbits = h.loc_jbits;
    db->max_probe = h.max_probe;
    db->overflow_keys = h.overflow_keys;
    {
        // most windows of one target, for the compact histogram keys
        std::vector<uint32_t> wb((size_t)h.n_targets + 1);
        if (cudaMemcpy(wb.data(), db->wbase.p, wb.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            mc_db_free(db);
            return fail(MC_ERR_CUDA, "mc_db_load: window bases");
        }
        for (uint32_t i = 0; i < h.n_targets; ++i)
            db->max_target_windows = std::max<uint64_t>(db->max_target_windows, wb[i + 1] - wb[i]);
    }
    db->has_table = true;
    db->dirty = false;
    ++db->epoch;
    cudaError_t e = cudaEventRecord(db->ready, db->stream);
    if (e != cudaSuccess) {
        mc_db_free(db);
        return cuda_fail(e, "mc_db_load");
    }
    *out = db;
    return MC_OK;
}

int mc_db_stats(const mc_db* db, mc_db_stats_t* out) {
    g_err[0] = 0;
    if (!db || !out) return fail(MC_ERR_ARG, "NULL argument");
    std::memset(out, 0, sizeof *out);
    out->n_targets = db->n_targets;
    out->n_windows = db->n_windows;
    out->n_pairs = db->n_pairs + db->pending_real;
    out->n_keys = db->n_keys;
    out->n_locations = db->n_kept;
    out->overflow_keys = db->overflow_keys;
    out->dropped_locations = out->n_pairs - db->n_kept;
    out->table_slots = db->has_table ? (1ull << db->fmt.log_t) : 0;
    out->max_probe = db->max_probe;
    out->device_bytes = held_bytes(db);
    out->load_factor = out->table_slots ? (double)db->n_keys / (double)out->table_slots : 0.0;
    out->finalized = db->dirty ? 0 : 1;
    out->max_depth = db->max_depth;
    out->loc_bytes = db->has_table ? mc::loc_bytes(db->loc_jbits) : 0;
    return MC_OK;
}

int mc_db_dump(const mc_db* db, uint64_t key_lo, uint64_t key_hi, uint64_t max_keys, uint64_t max_locs,
               uint32_t* keys, uint32_t* counts, uint64_t* locs, uint64_t* n_keys, uint64_t* n_locs) {
    g_err[0] = 0;
    if (!db || !n_keys || !n_locs) return fail(MC_ERR_ARG, "NULL argument");
    if (!db->has_table) return fail(MC_ERR_STATE, "mc_db_dump before mc_db_finalize");
    cudaStream_t s = db->stream;
    const uint64_t cap = std::max<uint64_t>(max_keys, 1);
    mc::Tmp<uint32_t> dkeys(db->mem, cap, s), dcnt(db->mem, cap, s);
    mc::Tmp<uint64_t> doff(db->mem, cap, s);
    mc::Tmp<unsigned long long> dn(db->mem, 1, s);
    if (!dkeys.ok() || !dcnt.ok() || !doff.ok() || !dn.ok()) return fail(MC_ERR_OOM, "dump: allocation failed");
    MC_CU(cudaMemsetAsync(dn.ptr, 0, 8, s));
    MC_CU(mc::dump_select((const uint64_t*)db->table.p, db->table_len, db->fmt, key_lo, key_hi, dkeys.ptr, doff.ptr,
                          dcnt.ptr, cap, dn.ptr, s));
    unsigned long long nsel = 0;
    MC_CU(cudaMemcpyAsync(&nsel, dn.ptr, 8, cudaMemcpyDeviceToHost, s));
    MC_CU(cudaStreamSynchronize(s));
    *n_keys = nsel;
    *n_locs = 0;
    if (nsel > max_keys) return fail(MC_ERR_CAPACITY, "dump: %llu features qualify", nsel);
    std::vector<uint32_t> hk(nsel), hc(nsel);
    std::vector<uint64_t> ho(nsel);
    if (nsel) {
        MC_CU(cudaMemcpyAsync(hk.data(), dkeys.ptr, nsel * 4, cudaMemcpyDeviceToHost, s));
        MC_CU(cudaMemcpyAsync(hc.data(), dcnt.ptr, nsel * 4, cudaMemcpyDeviceToHost, s));
        MC_CU(cudaMemcpyAsync(ho.data(), doff.ptr, nsel * 8, cudaMemcpyDeviceToHost, s));
        MC_CU(cudaStreamSynchronize(s));
    }
    std::vector<uint64_t> order(nsel);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](uint64_t x, uint64_t y) { return hk[x] < hk[y]; });
    uint64_t total = 0;
    for (uint64_t i = 0; i < nsel; ++i) total += hc[i];
    *n_locs = total;
    if (total > max_locs) return fail(MC_ERR_CAPACITY, "dump: %llu locations qualify", (unsigned long long)total);
    std::vector<uint64_t> src(nsel), dst(nsel);
    std::vector<uint32_t> cnt(nsel);
    uint64_t acc = 0;
    for (uint64_t i = 0; i < nsel; ++i) {
        uint64_t o = order[i];
        if (keys) keys[i] = hk[o];
        if (counts) counts[i] = hc[o];
        src[i] = ho[o];
        cnt[i] = hc[o];
        dst[i] = acc;
        acc += hc[o];
    }
    if (locs && total) {
        mc::Tmp<uint64_t> dsrc(db->mem, nsel, s), ddst(db->mem, nsel, s), dout(db->mem, total, s);
        mc::Tmp<uint32_t> dc(db->mem, nsel, s);
        if (!dsrc.ok() || !ddst.ok() || !dout.ok() || !dc.ok()) return fail(MC_ERR_OOM, "dump: allocation failed");
        MC_CU(cudaMemcpyAsync(dsrc.ptr, src.data(), nsel * 8, cudaMemcpyHostToDevice, s));
        MC_CU(cudaMemcpyAsync(ddst.ptr, dst.data(), nsel * 8, cudaMemcpyHostToDevice, s));
        MC_CU(cudaMemcpyAsync(dc.ptr, cnt.data(), nsel * 4, cudaMemcpyHostToDevice, s));
        MC_CU(mc::dump_gather(db->locs.p, db->loc_jbits, dsrc.ptr, dc.ptr, ddst.ptr, nsel, dout.ptr, s));
        MC_CU(cudaMemcpyAsync(locs, dout.ptr, total * 8, cudaMemcpyDeviceToHost, s));
        MC_CU(cudaStreamSynchronize(s));
    }
    return MC_OK;
}

int mc_window_offsets(const mc_db_params* params, uint32_t n_seq, const uint64_t* offs, uint64_t* win_offs,
                      void* stream) {
    g_err[0] = 0;
    int rc = check_params(params);
    if (rc) return rc;
    if (!win_offs || (n_seq && !offs)) return fail(MC_ERR_ARG, "NULL argument");
    mc::Mem mem;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        mem.a = g_alloc;
    }
    mc::Tmp<uint32_t> bad(mem, 1, (cudaStream_t)stream);
    if (!bad.ok()) return fail(MC_ERR_OOM, "allocation failed");
    MC_CU(cudaMemsetAsync(bad.ptr, 0, 4, (cudaStream_t)stream));
    MC_CU(mc::window_offsets(mem, sketch_params(params), n_seq, offs, win_offs, bad.ptr, (cudaStream_t)stream));
    return MC_OK;
}

int mc_sketch(const mc_db_params* params, uint32_t n_seq, const char* seq, const uint64_t* offs,
              const uint64_t* win_offs, uint64_t n_windows, uint32_t* sketch, uint32_t* counts, void* stream) {
    g_err[0] = 0;
    int rc = check_params(params);
    if (rc) return rc;
    if (n_windows == 0) return MC_OK;
    if (!seq || !offs || !win_offs || !sketch || !counts) return fail(MC_ERR_ARG, "NULL argument");
    MC_CU(mc::sketch_windows(sketch_params(params), n_seq, (const uint8_t*)seq, offs, win_offs, n_windows, sketch,
                             counts, (cudaStream_t)stream));
    return MC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------
// Batched classification, plans and the autotuner.

namespace {


mc::ClassifyQuery batch_query(const mc_db* db, const mc_classify_params* p, uint32_t n_q_cap,
                              const mc::BatchDesc* desc, const uint32_t* bhdr) {
    mc::ClassifyQuery q{};
    q.n_q = n_q_cap;
    q.m = p->max_candidates;
    q.hits_min = p->hits_min;
    q.band = p->lca_band_pct;
    q.max_insert = p->max_insert;
    q.status = (uint32_t*)db->status.p;
    q.batches = desc;
    q.bhdr = bhdr;
    return q;
}

int tuning_from(const mc_tuning* t, const mc::Tuning& dflt, mc::Tuning* out) {
    if (!t) {
        *out = dflt;
        return MC_OK;
    }
    mc::Tuning x = mc::DEFAULT_TUNING;
    if (t->hist_slots) x.hist_slots = t->hist_slots;
    if (t->probe_batch) x.probe_batch = t->probe_batch;
    if (t->gather_batch) x.gather_batch = t->gather_batch;
    if (t->lookup_warps) x.lookup_warps = t->lookup_warps;
    if (t->score_warps) x.score_warps = t->score_warps;
    if (t->wide_keys) x.wide_keys = t->wide_keys;
    if (t->score_mode) x.score_mode = t->score_mode;
    if (t->sort_max) x.sort_max = t->sort_max;
    if (!mc::tuning_valid(x)) return fail(MC_ERR_ARG, "tuning: a value is outside its allowed set");
    *out = x;
    return MC_OK;
}

mc_tuning to_public(const mc::Tuning& t) {
    return mc_tuning{t.hist_slots, t.probe_batch, t.gather_batch, t.lookup_warps,
                     t.score_warps, t.wide_keys,  t.score_mode,   t.sort_max};
}

// Host image of the batch header + descriptors (layout of ClassifyQuery's
// multi-batch form): bhdr words, then the descriptors at a 16-byte boundary.
size_t desc_offset(uint32_t n_batches) { return ((size_t)(n_batches + 3) * 4 + 15) & ~(size_t)15; }
size_t desc_bytes(uint32_t n_batches) { return desc_offset(n_batches) + (size_t)n_batches * sizeof(mc::BatchDesc); }

int fill_batches(uint32_t n_batches, const mc_batch* batches, unsigned char* img, uint64_t* total_out) {
    uint32_t* hdr = reinterpret_cast<uint32_t*>(img);
    mc::BatchDesc* d = reinterpret_cast<mc::BatchDesc*>(img + desc_offset(n_batches));
    uint64_t total = 0;
    hdr[0] = n_batches;
    for (uint32_t b = 0; b < n_batches; ++b) {
        const mc_batch& x = batches[b];
        if (x.n_queries && (!x.seq || !x.offs || !x.qoffs || !x.label || !x.hits))
            return fail(MC_ERR_ARG, "batch %u: NULL input or output pointer", b);
        hdr[2 + b] = (uint32_t)total;
        total += x.n_queries;
        if (total >= 0xFFFFFFFFull) return fail(MC_ERR_ARG, "batches: more than 2^32-2 queries in total");
        d[b] = mc::BatchDesc{(const uint8_t*)x.seq, x.offs, x.qoffs, x.label, x.hits, x.top_target};
    }
    hdr[1] = (uint32_t)total;
    hdr[2 + n_batches] = (uint32_t)total;
    *total_out = total;
    return MC_OK;
}

}  // namespace

struct mc_plan {
    const mc_db* db = nullptr;
    mc_classify_params params{};
    mc::Tuning tuning{};
    uint32_t max_batches = 0, max_queries = 0;
    DevBuf scratch, desc;
    mc::ClassifyScratch sc{};
    unsigned char* host = nullptr;  // pinned image of the descriptors
    cudaStream_t cap = nullptr;     // capture stream
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t copied = nullptr;   // the descriptor copy of the last run is done
    cudaEvent_t done = nullptr;     // the last run is done
    uint64_t epoch = ~0ull;
    int n_kernels = 0;
};

namespace {

void plan_drop_graph(mc_plan* p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
}

int plan_capture(mc_plan* p) {
    plan_drop_graph(p);
    const mc_db* db = p->db;
    const mc::ClassifyDb cdb = db_view(db);
    const uint32_t* bhdr = (const uint32_t*)p->desc.p;
    const mc::BatchDesc* d = (const mc::BatchDesc*)((unsigned char*)p->desc.p + desc_offset(p->max_batches));
    const mc::ClassifyQuery q = batch_query(db, &p->params, p->max_queries, d, bhdr);
    MC_CU(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    int nk = 0;
    cudaError_t e = mc::classify_enqueue(cdb, q, p->tuning, p->sc, p->cap, &nk);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(p->cap, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_fail(e != cudaSuccess ? e : e2, "mc_plan: capture");
    }
    p->graph = g;
    e = cudaGraphInstantiate(&p->exec, g, 0);
    if (e != cudaSuccess) {
        plan_drop_graph(p);
        return cuda_fail(e, "mc_plan: instantiate");
    }
    p->n_kernels = nk;
    p->epoch = db->epoch;
    return MC_OK;
}

}  // namespace

extern "C" {

int mc_db_set_tuning(mc_db* db, const mc_tuning* tuning) {
    g_err[0] = 0;
    if (!db) return fail(MC_ERR_ARG, "db is NULL");
    mc::Tuning t;
    int rc = tuning_from(tuning, mc::DEFAULT_TUNING, &t);
    if (rc) return rc;
    db->tuning = t;
    return MC_OK;
}

int mc_classify_batches(const mc_db* db, const mc_classify_params* params, const mc_tuning* tuning,
                        uint32_t n_batches, const mc_batch* batches, void* stream) {
    g_err[0] = 0;
    if (!db) return fail(MC_ERR_ARG, "db is NULL");
    int rc = check_cls(params);
    if (rc) return rc;
    if (!db->has_table) return fail(MC_ERR_STATE, "mc_classify_batches before mc_db_finalize");
    if (n_batches == 0) return MC_OK;
    if (!batches) return fail(MC_ERR_ARG, "batches is NULL");
    mc::Tuning t;
    if ((rc = tuning_from(tuning, db->tuning, &t))) return rc;
    std::vector<unsigned char> img(desc_bytes(n_batches));
    uint64_t total = 0;
    if ((rc = fill_batches(n_batches, batches, img.data(), &total))) return rc;
    if (total == 0) return MC_OK;
    cudaStream_t s = (cudaStream_t)stream;
    MC_CU(cudaStreamWaitEvent(s, db->ready, 0));
    const uint32_t lw = mc::classify_default_large_warps();
    const size_t sbytes = mc::classify_scratch_bytes((uint32_t)total, db->sp.s, lw);
    mc::Tmp<unsigned char> dev(db->mem, img.size(), s);
    mc::Tmp<unsigned char> scratch(db->mem, sbytes, s);
    if (!dev.ok() || !scratch.ok()) return fail(MC_ERR_OOM, "mc_classify_batches: allocation failed");
    // pageable source: the copy is staged before the call returns
    MC_CU(cudaMemcpyAsync(dev.ptr, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    const mc::ClassifyScratch sc = mc::classify_scratch_carve(scratch.ptr, (uint32_t)total, db->sp.s, lw);
    const mc::ClassifyQuery q = batch_query(db, params, (uint32_t)total,
                                            (const mc::BatchDesc*)(dev.ptr + desc_offset(n_batches)),
                                            (const uint32_t*)dev.ptr);
    MC_CU(mc::classify_enqueue(db_view(db), q, t, sc, s, nullptr));
    MC_CU(note_use(db, s));
    return MC_OK;
}

int mc_plan_create(const mc_db* db, const mc_classify_params* params, const mc_tuning* tuning,
                   uint32_t max_batches, uint32_t max_queries, mc_plan** out) {
    g_err[0] = 0;
    if (!db || !out) return fail(MC_ERR_ARG, "NULL argument");
    *out = nullptr;
    int rc = check_cls(params);
    if (rc) return rc;
    if (!db->has_table) return fail(MC_ERR_STATE, "mc_plan_create before mc_db_finalize");
    if (max_batches == 0 || max_queries == 0 || max_queries >= 0xFFFFFFFFu)
        return fail(MC_ERR_ARG, "mc_plan_create: max_batches and max_queries must be positive");
    mc_plan* p = new mc_plan();
    p->db = db;
    p->params = *params;
    p->max_batches = max_batches;
    p->max_queries = max_queries;
    if ((rc = tuning_from(tuning, db->tuning, &p->tuning))) {
        delete p;
        return rc;
    }
    auto bail = [&](int code) {
        mc_plan_free(p);
        return code;
    };
    mc_db* mdb = const_cast<mc_db*>(db);
    const uint32_t lw = mc::classify_default_large_warps();
    if (!grab(mdb, p->scratch, mc::classify_scratch_bytes(max_queries, db->sp.s, lw)) ||
        !grab(mdb, p->desc, desc_bytes(max_batches)))
        return bail(fail(MC_ERR_OOM, "mc_plan_create: allocation failed"));
    p->sc = mc::classify_scratch_carve((unsigned char*)p->scratch.p, max_queries, db->sp.s, lw);
    cudaError_t e;
    if ((e = cudaMallocHost(&p->host, desc_bytes(max_batches))) != cudaSuccess) {
        p->host = nullptr;
        return bail(cuda_fail(e, "mc_plan_create: pinned buffer"));
    }
    if ((e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking)) != cudaSuccess)
        return bail(cuda_fail(e, "mc_plan_create: stream"));
    if ((e = cudaEventCreateWithFlags(&p->copied, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming)) != cudaSuccess)
        return bail(cuda_fail(e, "mc_plan_create: event"));
    // the allocations above are stream-ordered on the database stream
    if ((e = cudaStreamSynchronize(db->stream)) != cudaSuccess) return bail(cuda_fail(e, "mc_plan_create"));
    if ((rc = plan_capture(p))) return bail(rc);
    *out = p;
    return MC_OK;
}

int mc_plan_run(mc_plan* p, uint32_t n_batches, const mc_batch* batches, void* stream) {
    g_err[0] = 0;
    if (!p) return fail(MC_ERR_ARG, "plan is NULL");
    if (n_batches && !batches) return fail(MC_ERR_ARG, "batches is NULL");
    if (n_batches > p->max_batches)
        return fail(MC_ERR_CAPACITY, "mc_plan_run: %u batches, plan holds %u", n_batches, p->max_batches);
    const mc_db* db = p->db;
    if (!db->has_table || db->dirty) return fail(MC_ERR_STATE, "mc_plan_run: database has pending additions");
    int rc;
    if (db->epoch != p->epoch && (rc = plan_capture(p))) return rc;
    // the previous run's descriptor copy must be done before the image is rewritten
    MC_CU(cudaEventSynchronize(p->copied));
    std::vector<unsigned char> img(desc_bytes(n_batches));
    uint64_t total = 0;
    if ((rc = fill_batches(n_batches, batches, img.data(), &total))) return rc;
    if (total > p->max_queries)
        return fail(MC_ERR_CAPACITY, "mc_plan_run: %llu queries, plan holds %u", (unsigned long long)total,
                    p->max_queries);
    // the plan's image layout has its descriptors after max_batches header words
    uint32_t* hdr = reinterpret_cast<uint32_t*>(p->host);
    std::memcpy(hdr, img.data(), (size_t)(n_batches + 3) * 4);
    std::memcpy(p->host + desc_offset(p->max_batches), img.data() + desc_offset(n_batches),
                (size_t)n_batches * sizeof(mc::BatchDesc));
    cudaStream_t s = (cudaStream_t)stream;
    MC_CU(cudaStreamWaitEvent(s, db->ready, 0));
    MC_CU(cudaMemcpyAsync(p->desc.p, p->host, desc_bytes(p->max_batches), cudaMemcpyHostToDevice, s));
    MC_CU(cudaEventRecord(p->copied, s));
    MC_CU(cudaGraphLaunch(p->exec, s));
    MC_CU(cudaEventRecord(p->done, s));
    mc::note_launches((uint64_t)p->n_kernels);
    MC_CU(note_use(db, s));
    return MC_OK;
}

int mc_plan_kernels(const mc_plan* p) { return p ? p->n_kernels : 0; }

void mc_plan_free(mc_plan* p) {
    if (!p) return;
    if (p->done) cudaEventSynchronize(p->done);
    plan_drop_graph(p);
    mc_db* mdb = const_cast<mc_db*>(p->db);
    release(mdb, p->scratch);
    release(mdb, p->desc);
    cudaStreamSynchronize(mdb->stream);
    if (p->host) cudaFreeHost(p->host);
    if (p->copied) cudaEventDestroy(p->copied);
    if (p->done) cudaEventDestroy(p->done);
    if (p->cap) cudaStreamDestroy(p->cap);
    cudaGetLastError();
    delete p;
}

int mc_autotune(const mc_db* db, const mc_classify_params* params, uint32_t n_batches, const mc_batch* batches,
                uint32_t reps, mc_tuning* best, mc_tuning_time* times, uint32_t max_times, uint32_t* n_times) {
    g_err[0] = 0;
    if (!db || !best) return fail(MC_ERR_ARG, "NULL argument");
    int rc = check_cls(params);
    if (rc) return rc;
    if (!db->has_table) return fail(MC_ERR_STATE, "mc_autotune before mc_db_finalize");
    if (n_batches == 0 || !batches || reps == 0) return fail(MC_ERR_ARG, "mc_autotune: no sample");
    std::vector<unsigned char> img(desc_bytes(n_batches));
    uint64_t total = 0;
    if ((rc = fill_batches(n_batches, batches, img.data(), &total))) return rc;
    if (total == 0 || total > mc::CLASSIFY_CHUNK)
        return fail(MC_ERR_ARG, "mc_autotune: sample must hold 1..%u queries", mc::CLASSIFY_CHUNK);
    cudaStream_t s = db->stream;
    MC_CU(cudaStreamWaitEvent(s, db->ready, 0));
    const uint32_t lw = mc::classify_default_large_warps();
    mc::Tmp<unsigned char> dev(db->mem, img.size(), s);
    mc::Tmp<unsigned char> scratch(db->mem, mc::classify_scratch_bytes((uint32_t)total, db->sp.s, lw), s);
    if (!dev.ok() || !scratch.ok()) return fail(MC_ERR_OOM, "mc_autotune: allocation failed");
    MC_CU(cudaMemcpyAsync(dev.ptr, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    const mc::ClassifyScratch sc = mc::classify_scratch_carve(scratch.ptr, (uint32_t)total, db->sp.s, lw);
    const mc::ClassifyQuery q = batch_query(db, params, (uint32_t)total,
                                            (const mc::BatchDesc*)(dev.ptr + desc_offset(n_batches)),
                                            (const uint32_t*)dev.ptr);
    mc::Tuning t;
    std::vector<mc::TuneRecord> rec;
    MC_CU(mc::classify_autotune(db_view(db), q, sc, reps, s, &t, &rec));
    *best = to_public(t);
    if (times)
        for (uint32_t i = 0; i < max_times && i < rec.size(); ++i)
            times[i] = mc_tuning_time{to_public(rec[i].t), rec[i].stage, rec[i].ms};
    if (n_times) *n_times = (uint32_t)rec.size();
    MC_CU(cudaStreamSynchronize(s));
    return MC_OK;
}

}  // extern "C"
