// Warp-cooperative minhash sketch of one window (Section 2, Section 5.2
// steps 1-3, Section 5.3).
//
// One warp computes the sketch of one window of up to 32*R bases:
//  1. lane l loads the R bases at window offsets R*l .. R*l+R-1 and encodes
//     them into 2-bit codes plus an invalid-base mask (Section 5.3: "3-bit"
//     A,C,G,T,N representation);
//  2. the codes of the next E = ceil((k-1)/R) lanes arrive by warp
//     shuffles, so lane l holds the R + E*R bases its k-mers need and forms
//     the k-mers starting at R*l .. R*l+R-1 (Section 5.3 does the same with
//     4-base loads and sub-warp shuffles; here the window start is any base,
//     the stride need not be a multiple of 4);
//  3. canonical code = min(forward, reverse complement), hashed by h1
//     (the reverse complement of all the lane's bases is formed once);
//  4. the s smallest distinct hashes (Section 2: repeated k-mers count
//     once) are selected by a cutoff + warp bitonic sort, with an exact
//     min-reduction fallback (see warp_sketch_multi).
// Lane i (< count) ends up holding the i-th smallest feature.  Several
// windows can be sketched together so that their dependency chains overlap.
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

// Encodes 4 bases packed little-endian in x (byte 0 = first base): code8 =
// their 2-bit codes, first base most significant; inv4 = 1 bit per invalid
// base, first base most significant.  A byte is a base iff (byte | 0x20)
// is one of a, c, g, t; each check is done on all four bytes at once.
__device__ __forceinline__ void encode4(uint32_t x, uint32_t& code8, uint32_t& inv4) {
    const uint32_t c = ((x >> 1) ^ (x >> 2)) & 0x03030303u;  // code of every byte
    code8 = (c * 0x40100401u) >> 24;                        // b0<<6 | b1<<4 | b2<<2 | b3
    // the only letter (lower case) with code c: 'a' + {0, 2, 6, 19}[c]
    const uint32_t hi = (c >> 1) & 0x01010101u;
    const uint32_t both = c & (c >> 1) & 0x01010101u;
    const uint32_t expect = 0x61616161u + (c << 1) + (hi << 1) + both * 11u;
    const uint32_t d = (x | 0x20202020u) ^ expect;            // zero byte <=> valid base
    uint32_t z = (d & 0x7F7F7F7Fu) + 0x7F7F7F7Fu;
    z = ~(z | d | 0x7F7F7F7Fu);                               // bit 7 of each zero byte
    const uint32_t valid = (((z >> 7) & 0x01010101u) * 0x08040201u) >> 24;  // b0<<3 | ... | b3
    inv4 = ~valid & 0xFu;
}

// Bitonic sort of one value per lane across the warp (ascending by lane),
// in mirror form: each merge stage of size k first pairs lane i with lane
// i ^ (k - 1), then with i ^ j for j = k/4 .. 1, and the lower lane of a
// pair always keeps the minimum (five lane-bit predicates in all).
__device__ __forceinline__ uint32_t warp_sort32(uint32_t v) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
        {
            const uint32_t u = __shfl_xor_sync(FULL_MASK, v, k - 1);
            v = (lane & (uint32_t)(k >> 1)) == 0 ? min(v, u) : max(v, u);
        }
#pragma unroll
        for (int j = k >> 2; j > 0; j >>= 1) {
            const uint32_t u = __shfl_xor_sync(FULL_MASK, v, j);
            v = (lane & (uint32_t)j) == 0 ? min(v, u) : max(v, u);
        }
    }
    return v;
}

// Computes the sketches of NW windows at once (independent dependency
// chains interleave).  Window w starts at base ws[w] of seq[w] (length
// L[w]; global memory, or shared memory when GLOBAL_SEQ is false); inactive
// windows yield count 0.  count[w] is warp-uniform; lane i < count[w] holds
// feature i of window w (ascending) in feature[w].  Requires 32*R >= w.
// cand: per-warp shared scratch of NW*32 words.
//
// Selection of the s smallest distinct hashes: a cutoff tau is chosen so
// that about 24 of the window's n_k hashes fall below it (all of them when
// n_k <= 32).  The hashes <= tau (at most 32 of them) are gathered one per
// lane, sorted by a warp bitonic network and de-duplicated.  If that gives
// at least s distinct values, or no valid hash lies above tau, they are
// exactly the s smallest distinct hashes.  Otherwise (a few percent of
// windows, and low-complexity windows) the exact fallback runs: s rounds of
// a warp min-reduction over locally sorted, de-duplicated lane lists.
template <int R, int NW, int KC = 0, bool GLOBAL_SEQ = true>
__device__ __forceinline__ void warp_sketch_multi(const uint8_t* const (&seq)[NW], const uint64_t (&L)[NW],
                                                  const uint64_t (&ws)[NW], const bool (&active)[NW],
                                                  const SketchParams& p, uint32_t* cand, uint32_t (&feature)[NW],
                                                  uint32_t (&count)[NW]) {
    constexpr int E_MAX = (15 + R - 1) / R;  // neighbours for k <= 16
    constexpr int T = R * (1 + E_MAX);       // bases held by a lane
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    const uint32_t k = KC ? (uint32_t)KC : p.k;  // k-mer length (compile-time when KC != 0)
    const uint32_t kmask_bits = 2 * k;
    const uint64_t cmask = (kmask_bits == 32) ? 0xFFFFFFFFull : ((1ull << kmask_bits) - 1);
    const uint64_t imask = (1ull << k) - 1;
    uint32_t h[NW][R];
    uint32_t vmask[NW];  // bit r: h[w][r] is a valid k-mer's hash
    bool fast[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t n_k = active[w] ? window_kmers(L[w], ws[w], p) : 0u;
        uint64_t lim = ws[w] + p.w;
        if (lim > L[w]) lim = L[w];
        if (!active[w]) lim = 0;
        // 1. load and encode R bases (bytes past the window's end read as 0,
        // an invalid base), four at a time
        uint32_t code = 0, inv = 0;
        const uint64_t b0 = ws[w] + (uint64_t)R * lane;
#pragma unroll
        for (int g = 0; g < R / 4; ++g) {
            uint32_t x = 0;
            if (GLOBAL_SEQ) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint64_t b = b0 + 4 * g + i;
                    const uint32_t c = b < lim ? (uint32_t)__ldg(seq[w] + b) : 0u;
                    x |= c << (8 * i);
                }
            } else {
                // staged bases: the aligned words holding bases bg .. bg+3 and a
                // funnel shift; a word is read only if it holds a base before
                // lim, so every read stays inside the staged range
                const uint64_t bg = b0 + 4 * g;
                if (bg < lim) {
                    const uintptr_t a = reinterpret_cast<uintptr_t>(seq[w] + bg);
                    const uint32_t sh = (uint32_t)(a & 3u);
                    const uint32_t* wp = reinterpret_cast<const uint32_t*>(a - sh);
                    const uint32_t lo = wp[0];
                    const uint32_t hi = (sh != 0 && bg + (4 - sh) < lim) ? wp[1] : 0u;
                    x = __funnelshift_r(lo, hi, 8 * sh);
                    const uint64_t nb = lim - bg;
                    if (nb < 4) x &= (1u << (8 * (uint32_t)nb)) - 1u;
                }
            }
            uint32_t c8, i4;
            encode4(x, c8, i4);
            code = (code << 8) | c8;
            inv = (inv << 4) | i4;
        }
        // 2. bases of the following lanes
        uint64_t comb = code, combinv = inv;
#pragma unroll
        for (int e = 1; e <= E_MAX; ++e) {
            comb = (comb << (2 * R)) | __shfl_down_sync(FULL_MASK, code, e);
            combinv = (combinv << R) | __shfl_down_sync(FULL_MASK, inv, e);
        }
        // 3. canonical k-mers and h1; the reverse complement of the lane's T
        // bases is formed once (reverse the 2-bit digits, complement), and
        // the k-mer starting at base r reads as its digits 2r .. 2r + 2k - 1
        vmask[w] = 0;
        uint64_t rcomb = __brevll(comb);
        rcomb = ((rcomb >> 1) & 0x5555555555555555ull) | ((rcomb & 0x5555555555555555ull) << 1);
        rcomb = ~rcomb >> (64 - 2 * T);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const uint32_t shift = (uint32_t)(T - r) - k;  // >= 0 since T >= R + k - 1
            const uint32_t fwd = (uint32_t)((comb >> (2 * shift)) & cmask);
            const bool bad = ((combinv >> shift) & imask) != 0;
            const bool ok = ((uint32_t)R * lane + r < n_k) && !bad;
            const uint32_t rc = (uint32_t)((rcomb >> (2 * r)) & cmask);
            h[w][r] = ok ? hash_h1(fwd < rc ? fwd : rc) : 0xFFFFFFFFu;
            vmask[w] |= (ok ? 1u : 0u) << r;
        }
        // 4. candidates below the cutoff, one per lane in cand[]
        // (any cutoff is correct; a fast reciprocal is plenty for aiming at ~24)
        const uint32_t tau = n_k <= 32 ? 0xFFFFFFFFu : __float2uint_rz(__fdividef(24.0f, (float)n_k) * 4294967296.0f);
        uint32_t cmine = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) cmine += (((vmask[w] >> r) & 1u) && h[w][r] <= tau) ? 1u : 0u;
        uint32_t pre = cmine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t x = __shfl_up_sync(FULL_MASK, pre, d);
            if ((int)lane >= d) pre += x;
        }
        const uint32_t C = __shfl_sync(FULL_MASK, pre, 31);
        const uint32_t Nv = __reduce_add_sync(FULL_MASK, (uint32_t)__popc(vmask[w]));
        pre -= cmine;
        fast[w] = C <= 32;
        if (fast[w]) {
            uint32_t o = pre;
#pragma unroll
            for (int r = 0; r < R; ++r)
                if (((vmask[w] >> r) & 1u) && h[w][r] <= tau) cand[w * 32 + o++] = h[w][r];
        }
        __syncwarp();
        if (fast[w]) {
            uint32_t v = lane < C ? cand[w * 32 + lane] : 0xFFFFFFFFu;
            v = warp_sort32(v);
            const uint32_t prev = __shfl_up_sync(FULL_MASK, v, 1);
            const bool fresh = lane < C && (lane == 0 || v != prev);
            const uint32_t nd = __ballot_sync(FULL_MASK, fresh);
            const uint32_t D = __popc(nd);
            fast[w] = D >= p.s || C == Nv;
            if (fast[w]) {
                if (D != C) {  // duplicates: compact the distinct values
                    __syncwarp();
                    if (fresh) cand[w * 32 + __popc(nd & lt)] = v;
                    __syncwarp();
                    v = cand[w * 32 + lane];
                }
                count[w] = D < p.s ? D : p.s;
                feature[w] = lane < count[w] ? v : 0u;
            }
        }
    }

    // exact fallback for the windows the cutoff did not settle
    uint32_t need = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) need |= (fast[w] ? 0u : 1u) << w;
    if (need == 0) return;
    int nv[NW];
    bool any_dup = false;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        nv[w] = 0;
        if (fast[w]) continue;
        // local sort + local de-duplication (valid entries become the first nv)
        nv[w] = __popc(vmask[w]);
        sort_small<R>(h[w]);
#pragma unroll
        for (int r = R - 1; r >= 1; --r) {
            if ((r < nv[w]) && (h[w][r] == h[w][r - 1])) {
                h[w][r] = 0xFFFFFFFFu;
                nv[w] -= 1;
                any_dup = true;
            }
        }
        count[w] = 0;
        feature[w] = 0;
    }
    if (__any_sync(FULL_MASK, any_dup)) {
#pragma unroll
        for (int w = 0; w < NW; ++w)
            if (!fast[w]) sort_small<R>(h[w]);
    }
    for (uint32_t it = 0; it < p.s; ++it) {
        uint32_t mine = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) mine |= (nv[w] > 0 ? 1u : 0u) << w;
        const uint32_t live = __reduce_or_sync(FULL_MASK, mine);
        if (live == 0) break;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            if (!((live >> w) & 1u)) continue;
            const bool has = nv[w] > 0;
            const uint32_t m = __reduce_min_sync(FULL_MASK, has ? h[w][0] : 0xFFFFFFFFu);
            const bool pop = has && (h[w][0] == m);
#pragma unroll
            for (int r = 0; r < R - 1; ++r) h[w][r] = pop ? h[w][r + 1] : h[w][r];
            h[w][R - 1] = pop ? 0xFFFFFFFFu : h[w][R - 1];
            nv[w] -= pop ? 1 : 0;
            if (lane == it) feature[w] = m;
            count[w] += 1;
        }
    }
}


// R for a window length: the warp covers 32*R >= w bases.
__host__ __device__ inline int sketch_r_for(uint32_t w) { return w <= 128 ? 4 : (w <= 256 ? 8 : 16); }

}  // namespace mc
