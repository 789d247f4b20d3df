// Shared device helpers of the sm_103a MetaCache-GPU kernels: k-mer hashing
// (h1) and table-slot hashing (h2), window counts, warp helpers and the
// parameters shared by the translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mc {

constexpr uint32_t FULL_MASK = 0xFFFFFFFFu;
constexpr uint32_t NO_TAXON = 0xFFFFFFFFu;
constexpr uint64_t SENTINEL_PAIR = ~0ull;  // marks an unused (feature, window) slot
constexpr uint64_t EMPTY_LOC = ~0ull;      // empty histogram slot (target 2^32-1 is never assigned)
constexpr int MAX_M = 8;
constexpr int MAX_S = 32;
constexpr int NUM_SMS_HINT = 152;

// Device status word values (ordered: a larger code wins with atomicMax).
constexpr uint32_t DEV_OK = 0;
constexpr uint32_t DEV_ERR_CAPACITY = 7;
constexpr uint32_t DEV_ERR_ARG = 1;

struct SketchParams {
    uint32_t k;       // k-mer length
    uint32_t s;       // sketch size
    uint32_t w;       // window length
    uint32_t stride;  // window stride
};

// ---------------------------------------------------------------- hashing
// h1: the lowbias32 mixer (C. Wellons, hash-prospector), a bijection on
// 32-bit words, applied to the canonical k-mer code (Section 4.1).
__host__ __device__ __forceinline__ uint32_t hash_h1(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// h2: MurmurHash3's 32-bit finalizer, a second bijection used only to place
// features in the table (Section 4.1: "to counteract the biased distribution
// of sketch values a second hash function h2 is applied").  Layout only: it
// does not change any result.
__host__ __device__ __forceinline__ uint32_t hash_h2(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85ebca6bU;
    x ^= x >> 13;
    x *= 0xc2b2ae35U;
    x ^= x >> 16;
    return x;
}

__host__ __device__ constexpr uint32_t mul_inverse(uint32_t a) {
    // Newton iteration for the inverse of an odd number modulo 2^32
    uint32_t x = a;
    for (int i = 0; i < 5; ++i) x *= 2u - a * x;
    return x;
}

__host__ __device__ __forceinline__ uint32_t unxorshift(uint32_t y, int s) {
    uint32_t x = y;
    for (int i = 0; i < 32 / s + 1; ++i) x = y ^ (x >> s);
    return x;
}

// Inverse of h2 (to report features in dumps).
__host__ __device__ __forceinline__ uint32_t hash_h2_inverse(uint32_t y) {
    y = unxorshift(y, 16);
    y *= mul_inverse(0xc2b2ae35U);
    y = unxorshift(y, 13);
    y *= mul_inverse(0x85ebca6bU);
    y = unxorshift(y, 16);
    return y;
}

// ------------------------------------------------------- feature table
// The condensed layout's feature table (Section 4.2 / 5.1: a single-value
// hash table from a feature to its bucket) holds one 8-byte word per slot.
// Features are placed by ordered linear probing in the order of h = h2(f):
// the home slot of h is its top log_t bits, and the word in slot s holds
//   count  (cbits bits, >= 1; 0 marks an empty slot),
//   disp   (TAB_DBITS bits: s - home),
//   low    (32 - log_t bits: the low bits of h),
//   offset (the remaining bits: the bucket's first location).
// The high bits of h are home = s - disp, so h is recovered exactly.
constexpr uint32_t TAB_DBITS = 6;
constexpr uint32_t TAB_MAX_DISP = (1u << TAB_DBITS) - 1;

struct TableFmt {
    uint32_t log_t;  // 1..32: slots = 2^log_t (plus padding)
    uint32_t cbits;  // bits of the count field
    __host__ __device__ __forceinline__ uint32_t lbits() const { return 32 - log_t; }
    __host__ __device__ __forceinline__ uint32_t obits() const { return 64 - cbits - TAB_DBITS - lbits(); }
    __host__ __device__ __forceinline__ uint64_t home(uint32_t h) const { return (uint64_t)(h >> lbits()); }
    __host__ __device__ __forceinline__ uint64_t pack(uint64_t off, uint32_t h, uint32_t disp, uint32_t cnt) const {
        const uint64_t low = (uint64_t)h & ((1ull << lbits()) - 1);
        return (((off << lbits() | low) << TAB_DBITS | disp) << cbits) | cnt;
    }
    __host__ __device__ __forceinline__ uint32_t count(uint64_t e) const {
        return (uint32_t)(e & ((1ull << cbits) - 1));
    }
    __host__ __device__ __forceinline__ uint32_t disp(uint64_t e) const {
        return (uint32_t)(e >> cbits) & TAB_MAX_DISP;
    }
    __host__ __device__ __forceinline__ uint64_t offset(uint64_t e) const {
        return e >> (cbits + TAB_DBITS + lbits());
    }
    // h2 value of the (non-empty) word e found in slot s
    __host__ __device__ __forceinline__ uint32_t key(uint64_t e, uint64_t s) const {
        const uint64_t low = (e >> (cbits + TAB_DBITS)) & ((1ull << lbits()) - 1);
        return (uint32_t)(((s - disp(e)) << lbits()) | low);
    }
};

// Bits of the count field for a bucket cap.
__host__ __device__ inline uint32_t count_bits(uint32_t cap) {
    uint32_t b = 1;
    while ((1ull << b) <= cap) ++b;
    return b;
}

// ------------------------------------------------------ windows, lanes
// Windows of a sequence of length L (k-mer starts 0, stride, 2 stride, ...).
__host__ __device__ __forceinline__ uint64_t num_windows(uint64_t L, uint32_t k, uint32_t stride) {
    return L < k ? 0 : (L - k + stride) / stride;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace mc
