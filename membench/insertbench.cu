// The build primitive of the paper's GPU database (Sections 5.1 and 5.3):
// every (feature, location) pair inserted into a hash table keyed by
// feature, with warp-aggregated atomics, each key holding at most `cap`
// locations.  This is a measurement aid of the benchmark, timed on the same
// pairs as the library's sort-based build so that the two can be compared;
// it is not part of the classification library.
//
// The pairs are the sketches of all windows: element e = w * s + i of
// sketch[] is feature i of window w (valid while i < counts[w]), with
// location w.  Two passes over them, each one kernel:
//   count: the lanes of a warp holding the same feature are grouped
//          (__match_any_sync); the group's leader claims the feature's slot
//          (linear probing, atomicCAS on the key) and adds the group size
//          to the slot's count (atomicAdd);
//   fill:  after the caller's exclusive scan of min(count, cap) over the
//          slots, the leader takes the group's places from the slot's
//          cursor (atomicAdd) and every lane whose place is below cap
//          writes its location at offset[slot] + place.
// Locations of a feature end up in arrival order (the cap keeps whichever
// arrive first), unlike the library's build, which keeps the cap smallest
// and orders every bucket.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

namespace {

thread_local char g_err[256] = "";

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr uint32_t EMPTY_KEY = 0xFFFFFFFFu;  // slot marker; the feature of that value is stored as 0xFFFFFFFE
constexpr int INS_THREADS = 256;

__device__ __forceinline__ uint32_t slot_of(uint32_t key, uint32_t log_slots) {
    // multiplicative hashing (Knuth): the top log_slots bits of key * 2^32/phi
    return (uint32_t)(((uint64_t)(key * 0x9E3779B1u) << 32) >> (64 - log_slots));
}

__device__ __forceinline__ bool pair_at(const uint32_t* __restrict__ sketch, const uint32_t* __restrict__ counts,
                                        uint64_t n, uint32_t s, uint64_t e, uint32_t& key) {
    if (e >= n) return false;
    const uint64_t w = e / s;
    if ((uint32_t)(e - w * s) >= counts[w]) return false;
    key = sketch[e];
    if (key == EMPTY_KEY) key = EMPTY_KEY - 1;
    return true;
}

__global__ void __launch_bounds__(INS_THREADS) k_insert_count(const uint32_t* __restrict__ sketch,
                                                              const uint32_t* __restrict__ counts, uint64_t n,
                                                              uint32_t s, uint32_t* keys, uint32_t* cnt,
                                                              uint32_t log_slots, uint32_t max_probe,
                                                              uint32_t* err) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t mask = (1u << log_slots) - 1u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); e0 < n; e0 += stride) {
        uint32_t key = EMPTY_KEY;
        const bool valid = pair_at(sketch, counts, n, s, e0 + lane, key);
        const uint32_t peers = __match_any_sync(FULL, valid ? key : EMPTY_KEY);
        if (valid && lane == (uint32_t)(__ffs(peers) - 1)) {
            uint32_t slot = slot_of(key, log_slots);
            uint32_t p = 0;
            for (; p <= max_probe; ++p) {
                const uint32_t old = atomicCAS(keys + slot, EMPTY_KEY, key);
                if (old == EMPTY_KEY || old == key) {
                    atomicAdd(cnt + slot, (uint32_t)__popc(peers));
                    break;
                }
                slot = (slot + 1) & mask;
            }
            if (p > max_probe) atomicOr(err, 1u);
        }
    }
}

__global__ void __launch_bounds__(INS_THREADS) k_insert_fill(const uint32_t* __restrict__ sketch,
                                                             const uint32_t* __restrict__ counts, uint64_t n,
                                                             uint32_t s, const uint32_t* __restrict__ keys,
                                                             const uint64_t* __restrict__ offset, uint32_t* cursor,
                                                             uint32_t* __restrict__ vals, uint32_t cap,
                                                             uint32_t log_slots, uint32_t max_probe, uint32_t* err) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t mask = (1u << log_slots) - 1u;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e0 = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); e0 < n; e0 += stride) {
        const uint64_t e = e0 + lane;
        uint32_t key = EMPTY_KEY;
        const bool valid = pair_at(sketch, counts, n, s, e, key);
        const uint32_t peers = __match_any_sync(FULL, valid ? key : EMPTY_KEY);
        const uint32_t leader = (uint32_t)(__ffs(peers) - 1);
        uint32_t base = 0, slot = 0;
        if (valid && lane == leader) {
            slot = slot_of(key, log_slots);
            uint32_t p = 0;
            for (; p <= max_probe && keys[slot] != key; ++p) slot = (slot + 1) & mask;
            if (p > max_probe) {
                atomicOr(err, 2u);
                slot = FULL;
            } else {
                base = atomicAdd(cursor + slot, (uint32_t)__popc(peers));
            }
        }
        base = __shfl_sync(FULL, base, leader);
        slot = __shfl_sync(FULL, slot, leader);
        const uint32_t place = base + (uint32_t)__popc(peers & lt);
        if (valid && slot != FULL && place < cap) vals[offset[slot] + place] = (uint32_t)(e / s);
    }
}

int fail(cudaError_t e, const char* what) {
    snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
    return 2;
}

// Times one launch of `launch` on stream s with CUDA events, in ms.
template <class F>
int timed(cudaStream_t s, F launch, double* ms, const char* what) {
    cudaEvent_t a, b;
    cudaError_t e;
    if ((e = cudaEventCreate(&a)) != cudaSuccess) return fail(e, what);
    if ((e = cudaEventCreate(&b)) != cudaSuccess) {
        cudaEventDestroy(a);
        return fail(e, what);
    }
    cudaEventRecord(a, s);
    launch();
    e = cudaGetLastError();
    cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float x = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return fail(e, what);
    *ms = x;
    return 0;
}

uint32_t grid_for(uint64_t n) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t want = (n + INS_THREADS - 1) / INS_THREADS;
    const uint64_t cap = (uint64_t)sms * 8;
    return (uint32_t)(want < cap ? (want ? want : 1) : cap);
}

}  // namespace

// Message of the last failed insert call on this thread.
extern "C" const char* membench_insert_last_error(void) { return g_err; }

// Count pass.  keys (2^log_slots, all 0xFFFFFFFF; log_slots <= 31) and cnt
// (2^log_slots, all 0) are device buffers of the caller; *ms receives the
// kernel time.  Returns 0, 1 (bad argument or a probe longer than
// max_probe) or 2 (CUDA error); membench_insert_last_error has the message.
extern "C" int membench_insert_count(const uint32_t* sketch, const uint32_t* counts, uint64_t n_windows,
                                     uint32_t s, uint32_t log_slots, uint32_t max_probe, uint32_t* keys,
                                     uint32_t* cnt, uint32_t* err, void* stream, double* ms) {
    if (!sketch || !counts || !keys || !cnt || !err || !ms || s == 0 || log_slots < 1 || log_slots > 31) {
        snprintf(g_err, sizeof(g_err), "membench_insert_count: bad argument");
        return 1;
    }
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t n = n_windows * s;
    int rc = timed(
        st, [&] { k_insert_count<<<grid_for(n), INS_THREADS, 0, st>>>(sketch, counts, n, s, keys, cnt, log_slots,
                                                                     max_probe, err); },
        ms, "membench_insert_count");
    if (rc) return rc;
    uint32_t h = 0;
    cudaError_t e = cudaMemcpy(&h, err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(e, "membench_insert_count");
    if (h) {
        snprintf(g_err, sizeof(g_err), "membench_insert_count: a probe passed %u slots", max_probe);
        return 1;
    }
    return 0;
}

// Fill pass: offset (2^log_slots, exclusive scan of min(cnt, cap)), cursor
// (2^log_slots, all 0) and vals (sum of min(cnt, cap) words) are device
// buffers of the caller.  Same returns as membench_insert_count.
extern "C" int membench_insert_fill(const uint32_t* sketch, const uint32_t* counts, uint64_t n_windows, uint32_t s,
                                    uint32_t log_slots, uint32_t max_probe, const uint32_t* keys,
                                    const uint64_t* offset, uint32_t* cursor, uint32_t* vals, uint32_t cap,
                                    uint32_t* err, void* stream, double* ms) {
    if (!sketch || !counts || !keys || !offset || !cursor || !vals || !err || !ms || s == 0 || log_slots < 1 ||
        log_slots > 31) {
        snprintf(g_err, sizeof(g_err), "membench_insert_fill: bad argument");
        return 1;
    }
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const uint64_t n = n_windows * s;
    int rc = timed(
        st, [&] { k_insert_fill<<<grid_for(n), INS_THREADS, 0, st>>>(sketch, counts, n, s, keys, offset, cursor, vals,
                                                                    cap, log_slots, max_probe, err); },
        ms, "membench_insert_fill");
    if (rc) return rc;
    uint32_t h = 0;
    cudaError_t e = cudaMemcpy(&h, err, 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(e, "membench_insert_fill");
    if (h) {
        snprintf(g_err, sizeof(g_err), "membench_insert_fill: a key was not found within %u slots", max_probe);
        return 1;
    }
    return 0;
}
