// mc_classify_noalloc: read classification that allocates no device memory.
//
// Some callers cannot allocate while they classify: a serving process whose
// device memory is entirely reserved by another allocator (a framework that
// pre-allocates the GPU up front), or a latency-critical loop that must not
// take the driver's allocation path (and its implicit synchronisation) on
// every request.  mc_classify gets its per-call scratch from the allocator
// hook; this entry point instead uses one fixed scratch area compiled into
// the library: a file-scope __device__ array that every GPU which loads the
// library holds until the process exits.  The caller still supplies inputs
// and outputs.
#include <cstdint>
#include <mutex>

#include "mc_internal.h"

namespace {

// The fixed scratch area (MC_NOALLOC_SCRATCH_BYTES per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[MC_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.  In host code the
// array's name is only a host-side stand-in, so kernels must get this
// address instead.  The cache is never invalidated: the address stays valid
// for the life of the device's primary context (a cudaDeviceReset after the
// first call is not supported).
int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mc::report_error(MC_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return mc::report_error(MC_ERR_CAPACITY, "device index %d too large", dev);
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return mc::report_error(MC_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                                    cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return MC_OK;
}

}  // namespace

extern "C" int mc_classify_noalloc(const mc_db* db, const mc_classify_params* params, uint32_t n_seq,
                                   const char* seq, const uint64_t* offs, uint32_t n_queries, const uint32_t* qoffs,
                                   uint32_t* label, uint32_t* hits, uint32_t* top_target, void* stream) {
    (void)n_seq;
    if (n_queries > MC_NOALLOC_MAX_QUERIES)
        return mc::report_error(MC_ERR_CAPACITY,
                                "mc_classify_noalloc takes at most %u queries per call (got %u); split the batch",
                                (unsigned)MC_NOALLOC_MAX_QUERIES, n_queries);
    cudaStream_t s = (cudaStream_t)stream;
    mc::ClassifyDb cdb;
    mc::ClassifyQuery q;
    int rc = mc::classify_prepare(db, params, seq, offs, n_queries, qoffs, label, hits, top_target, s, &cdb, &q);
    if (rc != MC_OK || n_queries == 0) return rc;
    const size_t need = mc::classify_noalloc_bytes(n_queries, cdb.sp.s);
    if (need > MC_NOALLOC_SCRATCH_BYTES)
        return mc::report_error(MC_ERR_CAPACITY, "mc_classify_noalloc needs %zu scratch bytes, has %zu", need,
                                (size_t)MC_NOALLOC_SCRATCH_BYTES);
    void* scratch = nullptr;
    rc = scratch_address(&scratch);
    if (rc != MC_OK) return rc;
    cudaError_t e = mc::classify_launch_noalloc(cdb, q, mc::db_tuning(db), static_cast<unsigned char*>(scratch),
                                                MC_NOALLOC_SCRATCH_BYTES, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return mc::report_error(MC_ERR_CUDA, "mc_classify_noalloc launch: %s", cudaGetErrorString(e));
    }
    return mc::classify_done(db, s);
}
