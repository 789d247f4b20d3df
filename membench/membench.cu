// Random-access read bandwidth of the device: the roofline of the feature
// table probes and bucket gathers of classification, which read 16-32 bytes
// at random positions.  Every thread reads items of `width` bytes (16 or 32,
// aligned) at uniformly random positions of a buffer much larger than L2,
// several reads in flight, and folds them into one word so that no read can
// be dropped.
//
// A measurement aid of the benchmark, built into its own library
// (libmembench.so); it is not part of the classification library's ABI.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

namespace {

thread_local char g_err[256] = "";
constexpr int NUM_SMS_HINT = 152;

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    // splitmix64 finaliser (Steele, Lea, Flood 2014)
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

constexpr int MB_THREADS = 256;
constexpr int MB_INFLIGHT = 8;

// MOD: index by 64-bit remainder (slower to compute, which spaces the
// requests out) instead of a multiply-high.
template <int WIDTH, bool MOD>
__global__ void __launch_bounds__(MB_THREADS) k_random_read(const uint4* __restrict__ buf, uint64_t n_items,
                                                            uint64_t per_thread, uint64_t seed,
                                                            uint32_t* __restrict__ out) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (uint64_t i = 0; i < per_thread; i += MB_INFLIGHT) {
        uint4 v[MB_INFLIGHT][WIDTH / 16];
#pragma unroll
        for (int j = 0; j < MB_INFLIGHT; ++j) {
            const uint64_t h = mix64(seed ^ (tid * per_thread + i + j));
            const uint64_t item = MOD ? h % n_items : __umul64hi(h, n_items);  // uniform in [0, n_items)
#pragma unroll
            for (int q = 0; q < WIDTH / 16; ++q) v[j][q] = __ldg(buf + item * (WIDTH / 16) + q);
        }
#pragma unroll
        for (int j = 0; j < MB_INFLIGHT; ++j)
#pragma unroll
            for (int q = 0; q < WIDTH / 16; ++q) acc ^= v[j][q].x ^ v[j][q].y ^ v[j][q].z ^ v[j][q].w;
    }
    out[tid] = acc;
}

}  // namespace

// Message of the last failed call on this thread.
extern "C" const char* membench_last_error(void) { return g_err; }

// n_reads reads of `width` bytes (16 or 32) at uniformly random positions of
// a fresh device buffer of buf_bytes (>= 1 MiB; take it much larger than
// L2), 8 reads in flight per thread, at 16, 32 and 64 warps per SM and two
// index generators, each timed with CUDA events after a warm-up launch.
// *gbs receives the best width x reads / time in GB/s (more requests in
// flight can lower random DRAM throughput, so the best shape is the
// roofline).  The buffer comes from cudaMallocAsync on `stream` and is freed
// before the call returns (synchronises `stream`).  Returns 0, 1 for a bad
// argument, 6 for a CUDA error (message: membench_last_error).
extern "C" int membench_random_read(uint64_t buf_bytes, uint32_t width, uint64_t n_reads, void* stream,
                                    double* gbs) {
    if (!gbs || (width != 16 && width != 32) || buf_bytes < (1u << 20) || n_reads == 0) {
        snprintf(g_err, sizeof g_err, "membench_random_read: width 16 or 32, buffer >= 1 MiB, reads > 0");
        return 1;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = NUM_SMS_HINT;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t max_threads = (uint64_t)sms * 64 * 32;
    const uint64_t n_items = buf_bytes / width;
    void* buf = nullptr;
    uint32_t* out = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, n_items * width, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&out, max_threads * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0x5A, n_items * width, s);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    // the best of two index generators x three occupancies (16, 32, 64
    // warps per SM): too many requests in flight lower random-access
    // throughput, so the peak is taken over these shapes
    double best = 0;
    for (int mod = 0; mod < 2 && e == cudaSuccess; ++mod) {
        for (int wps = 16; wps <= 64 && e == cudaSuccess; wps *= 2) {
            const uint64_t threads = (uint64_t)sms * wps * 32;
            const uint64_t per_thread =
                std::max<uint64_t>(MB_INFLIGHT, (n_reads / threads + MB_INFLIGHT - 1) / MB_INFLIGHT * MB_INFLIGHT);
            auto k = width == 16 ? (mod ? k_random_read<16, true> : k_random_read<16, false>)
                                 : (mod ? k_random_read<32, true> : k_random_read<32, false>);
            const uint32_t grid = (uint32_t)(threads / MB_THREADS);
            k<<<grid, MB_THREADS, 0, s>>>((const uint4*)buf, n_items, per_thread, 1, out);  // warm-up
            cudaEventRecord(a, s);
            k<<<grid, MB_THREADS, 0, s>>>((const uint4*)buf, n_items, per_thread, 2, out);
            cudaEventRecord(b, s);
            float ms = 0;
            e = cudaEventSynchronize(b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess && ms > 0) best = std::max(best, (double)threads * per_thread * width / (ms * 1e-3) / 1e9);
        }
    }
    if (buf) cudaFreeAsync(buf, s);
    if (out) cudaFreeAsync(out, s);
    cudaStreamSynchronize(s);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        snprintf(g_err, sizeof g_err, "membench_random_read: %s", cudaGetErrorString(e));
        return 6;
    }
    *gbs = best;
    return 0;
}
