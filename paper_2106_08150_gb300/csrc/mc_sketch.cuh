// Warp-cooperative minhash sketch of one window (Section 2, Section 4.2
// steps 1-3, Section 4.3).
//
// One warp computes the sketch of one window of up to 32*R bases:
//  1. lane l loads the R bases at window offsets R*l .. R*l+R-1 and encodes
//     them into 2-bit codes plus an invalid-base mask (Section 4.3: "3-bit"
//     A,C,G,T,N representation);
//  2. the codes of the next E = ceil((k-1)/R) lanes arrive by warp
//     shuffles, so lane l holds the R + E*R bases its k-mers need and forms
//     the k-mers starting at R*l .. R*l+R-1 (Section 4.3 does the same with
//     4-base loads and sub-warp shuffles; here the window start is any base,
//     the stride need not be a multiple of 4);
//  3. canonical code = min(forward, reverse complement), hashed by h1;
//  4. the s smallest distinct hashes are extracted with s rounds of a warp
//     min-reduction (redux.sync) over the lanes' locally sorted, locally
//     de-duplicated lists: each round pops the minimum from every lane that
//     holds it, so repeated k-mers count once (Section 2).
// Lane i (< count) ends up holding the i-th smallest feature.
#pragma once

#include "mc_common.cuh"

namespace mc {

template <int R>
__device__ __forceinline__ void sort_small(uint32_t (&h)[R]) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
#pragma unroll
        for (int j = 0; j < R - 1 - i; ++j) {
            uint32_t a = h[j], b = h[j + 1];
            h[j] = min(a, b);
            h[j + 1] = max(a, b);
        }
    }
}

// Number of k-mer starts of the window that starts at `ws` in a sequence
// of length L (the window exists, i.e. ws + k <= L).
__device__ __forceinline__ uint32_t window_kmers(uint64_t L, uint64_t ws, const SketchParams& p) {
    uint64_t last = ws + p.w - p.k;
    if (last > L - p.k) last = L - p.k;
    return (uint32_t)(last - ws + 1);
}

// Computes the sketch of the window starting at base `ws` of `seq` (length
// L).  Returns the number of features (warp-uniform); lane i < count holds
// feature i (ascending) in `feature`.  Requires 32*R >= w.
template <int R>
__device__ __forceinline__ uint32_t warp_sketch(const uint8_t* __restrict__ seq, uint64_t L, uint64_t ws,
                                                const SketchParams& p, uint32_t& feature) {
    constexpr int E_MAX = (15 + R - 1) / R;  // neighbours for k <= 16
    const uint32_t lane = lane_id();
    const uint32_t n_k = window_kmers(L, ws, p);
    uint64_t lim = ws + p.w;
    if (lim > L) lim = L;

    // 1. load and encode R bases
    uint32_t code = 0, inv = 0;
    const uint64_t b0 = ws + (uint64_t)R * lane;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        uint64_t b = b0 + i;
        uint32_t c = (b < lim) ? (uint32_t)__ldg(seq + b) : 0u;
        uint32_t ok = (b < lim) ? base_valid(c) : 0u;
        code = (code << 2) | base_code(c);
        inv = (inv << 1) | (ok ^ 1u);
    }

    // 2. bases of the following lanes
    uint64_t comb = code, combinv = inv;
#pragma unroll
    for (int e = 1; e <= E_MAX; ++e) {
        uint32_t c2 = __shfl_down_sync(FULL_MASK, code, e);
        uint32_t i2 = __shfl_down_sync(FULL_MASK, inv, e);
        comb = (comb << (2 * R)) | c2;
        combinv = (combinv << R) | i2;
    }
    constexpr int T = R * (1 + E_MAX);  // bases held by this lane

    // 3. canonical k-mers and h1
    uint32_t h[R];
    int nv = 0;
    const uint32_t kmask_bits = 2 * p.k;
    const uint64_t cmask = (kmask_bits == 32) ? 0xFFFFFFFFull : ((1ull << kmask_bits) - 1);
    const uint64_t imask = (1ull << p.k) - 1;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const uint32_t shift = (uint32_t)(T - r) - p.k;  // T - r - k >= 0 since T >= R + k - 1
        uint32_t fwd = (uint32_t)((comb >> (2 * shift)) & cmask);
        bool bad = ((combinv >> shift) & imask) != 0;
        uint32_t pos = (uint32_t)R * lane + r;
        bool ok = (pos < n_k) && !bad;
        uint32_t rc = revcomp_code(fwd, p.k);
        uint32_t canon = fwd < rc ? fwd : rc;
        h[r] = ok ? hash_h1(canon) : 0xFFFFFFFFu;
        nv += ok ? 1 : 0;
    }

    // 4. local sort + local de-duplication (valid entries are the first nv)
    sort_small<R>(h);
    int ndup = 0;
#pragma unroll
    for (int r = R - 1; r >= 1; --r) {
        bool dup = (r < nv) && (h[r] == h[r - 1]);
        if (dup) { h[r] = 0xFFFFFFFFu; ++ndup; }
    }
    if (__any_sync(FULL_MASK, ndup > 0)) {
        sort_small<R>(h);
        nv -= ndup;
    }

    // s rounds of warp-wide minimum extraction
    uint32_t cnt = 0;
    feature = 0;
    for (uint32_t it = 0; it < p.s; ++it) {
        bool has = nv > 0;
        if (!__any_sync(FULL_MASK, has)) break;
        uint32_t head = has ? h[0] : 0xFFFFFFFFu;
        uint32_t m = __reduce_min_sync(FULL_MASK, head);
        bool pop = has && (h[0] == m);
#pragma unroll
        for (int r = 0; r < R - 1; ++r) h[r] = pop ? h[r + 1] : h[r];
        h[R - 1] = pop ? 0xFFFFFFFFu : h[R - 1];
        nv -= pop ? 1 : 0;
        if (lane == it) feature = m;
        ++cnt;
    }
    return cnt;
}

// R for a window length: the warp covers 32*R >= w bases.
__host__ __device__ inline int sketch_r_for(uint32_t w) { return w <= 128 ? 4 : (w <= 256 ? 8 : 16); }

}  // namespace mc
