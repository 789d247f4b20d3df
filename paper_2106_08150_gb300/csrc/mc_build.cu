// Database build kernels (Section 4.1 build phase, Section 5.1 GPU hash
// tables, Section 5.2 build pipeline) for sm_103a.
//
// GB300 design.  The paper inserts each (feature, location) pair into a
// multi-bucket hash table with warp-aggregated atomics.  Here the build is
// organised around streaming HBM passes instead of random-sector updates:
//   1. sketch + emit: one warp per window computes its sketch (shared with
//      the query path, mc_sketch.cuh) and writes (h2(feature) << 32 |
//      global window) pairs in window order;
//   2. a stable LSD radix sort (4 single-pass digits of 8 bits over the
//      upper word) groups the pairs by feature while keeping them in window order,
//      which is (target, window) order, so every bucket comes out sorted;
//   3. finalize keeps the first `cap` pairs of each feature (Section 4.1:
//      at most 254 locations per feature; the smallest are kept, as in the
//      CPU version that inserts in ascending order), converts global windows
//      to (target, window) locations, and lays out the condensed layout of
//      Section 5.1: one contiguous location array plus a feature table;
//   4. the feature table is an ordered linear-probing table built without
//      atomics: features arrive sorted by h2, so slot(k) = max(home(k),
//      slot(k-1)+1) = k + max_{k'<=k}(home(k') - k'), a max-scan.
// Every step reads and writes HBM in coalesced streams; the only random
// accesses of the whole database life are the lookups of the query path.
#include <atomic>
#include <cstdio>
#include <vector>

#include "mc_internal.h"
#include "mc_sketch.cuh"

namespace mc {

namespace {

constexpr int BT = 256;  // threads of the streaming kernels
constexpr int NWARP = BT / 32;

inline uint32_t grid_for(uint64_t tiles, uint32_t per_sm = 8) {
    uint64_t g = (uint64_t)NUM_SMS_HINT * per_sm;
    if (tiles < g) g = tiles;
    return (uint32_t)(g ? g : 1);
}

struct OpSum {
    __device__ __forceinline__ uint64_t operator()(uint64_t a, uint64_t b) const { return a + b; }
};
struct OpMaxU {
    __device__ __forceinline__ uint64_t operator()(uint64_t a, uint64_t b) const { return a > b ? a : b; }
};
struct OpMaxI {
    __device__ __forceinline__ int64_t operator()(int64_t a, int64_t b) const { return a > b ? a : b; }
};

template <class T, class Op>
__device__ __forceinline__ T warp_inclusive(T v, Op op) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = __shfl_up_sync(FULL_MASK, v, d);
        if ((int)lane_id() >= d) v = op(v, o);
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (BT threads).  Returns
// the exclusive prefix; *total receives the block aggregate.  `sm` needs
// NWARP entries.  Contains two __syncthreads.
template <class T, class Op>
__device__ __forceinline__ T block_exclusive(T v, T identity, Op op, T* sm, T* total) {
    T inc = warp_inclusive(v, op);
    const int w = threadIdx.x >> 5;
    const int l = lane_id();
    if (l == 31) sm[w] = inc;
    __syncthreads();
    T warp_pre = identity, tot = identity;
#pragma unroll
    for (int i = 0; i < NWARP; ++i) {
        T x = sm[i];
        if (i < w) warp_pre = op(warp_pre, x);
        tot = op(tot, x);
    }
    T ex = __shfl_up_sync(FULL_MASK, inc, 1);
    if (l == 0) ex = identity;
    *total = tot;
    __syncthreads();
    return op(warp_pre, ex);
}

template <class T, class Op>
__device__ __forceinline__ T block_reduce(T v, T identity, Op op, T* sm) {
    T tot;
    block_exclusive(v, identity, op, sm, &tot);
    return tot;
}

// ------------------------------------------------------------------ scan
constexpr int SCAN_ITEMS = 8;
constexpr uint64_t SCAN_TILE = (uint64_t)BT * SCAN_ITEMS;

__global__ void __launch_bounds__(BT) k_scan_tile_sums(const uint64_t* __restrict__ in, uint64_t n,
                                                       uint64_t* __restrict__ sums, uint64_t n_tiles) {
    __shared__ uint64_t sm[NWARP];
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        uint64_t base = tile * SCAN_TILE, acc = 0;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            uint64_t e = base + (uint64_t)i * BT + threadIdx.x;
            if (e < n) acc += in[e];
        }
        uint64_t tot = block_reduce(acc, (uint64_t)0, OpSum(), sm);
        if (threadIdx.x == 0) sums[tile] = tot;
    }
}

// Exclusive scan of each tile with its prefix (tile_pre, or 0 if null).
// The element of round i, thread t is base + i*BT + t (sequential order).
__global__ void __launch_bounds__(BT) k_scan_downsweep(const uint64_t* in, uint64_t* out, uint64_t n,
                                                       const uint64_t* __restrict__ tile_pre, uint64_t n_tiles,
                                                       uint64_t* total) {
    __shared__ uint64_t sm[NWARP];
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        uint64_t base = tile * SCAN_TILE;
        uint64_t carry = tile_pre ? tile_pre[tile] : 0;
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            uint64_t e = base + (uint64_t)i * BT + threadIdx.x;
            uint64_t v = e < n ? in[e] : 0;
            uint64_t tot;
            uint64_t ex = block_exclusive(v, (uint64_t)0, OpSum(), sm, &tot);
            if (e < n) out[e] = carry + ex;
            carry += tot;
        }
        if (tile == n_tiles - 1 && threadIdx.x == 0 && total) *total = carry;
    }
}

}  // namespace

cudaError_t scan_exclusive_sum(const Mem& mem, const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(uint64_t), s);
    uint64_t n_tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (n_tiles == 1) {
        MC_LAUNCH("scan_downsweep", s, k_scan_downsweep<<<1, BT, 0, s>>>(in, out, n, nullptr, 1, out + n));
        return cudaGetLastError();
    }
    Tmp<uint64_t> sums(mem, n_tiles + 1, s);
    if (!sums.ok()) return cudaErrorMemoryAllocation;
    MC_LAUNCH("scan_tile_sums", s, k_scan_tile_sums<<<grid_for(n_tiles), BT, 0, s>>>(in, n, sums.ptr, n_tiles));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_exclusive_sum(mem, sums.ptr, sums.ptr, n_tiles, s);
    if (e != cudaSuccess) return e;
    MC_LAUNCH("scan_downsweep", s, k_scan_downsweep<<<grid_for(n_tiles), BT, 0, s>>>(in, out, n, sums.ptr, n_tiles, out + n));
    return cudaGetLastError();
}

// ------------------------------------------------------ window offsets
namespace {
__global__ void k_window_counts(const uint64_t* __restrict__ offs, uint32_t n, uint32_t k, uint32_t stride,
                                uint64_t* __restrict__ cnt, uint32_t* bad) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t a = offs[i], b = offs[i + 1];
        if (b < a) {
            atomicMax(bad, 1u);
            cnt[i] = 0;
        } else {
            cnt[i] = num_windows(b - a, k, stride);
        }
    }
}
}  // namespace

cudaError_t window_offsets(const Mem& mem, const SketchParams& p, uint32_t n_seq, const uint64_t* offs,
                           uint64_t* win_offs, uint32_t* bad_offs, cudaStream_t s) {
    if (n_seq > 0) {
        MC_LAUNCH("window_counts", s, k_window_counts<<<grid_for((n_seq + BT - 1) / BT), BT, 0, s>>>(offs, n_seq, p.k, p.stride, win_offs,
                                                                         bad_offs));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return scan_exclusive_sum(mem, win_offs, win_offs, n_seq, s);
}

// ---------------------------------------------------------------- sketch
namespace {
constexpr uint32_t WINDOWS_PER_TASK = 16;
constexpr int SK_NW = 2;  // windows sketched together by a warp

// One warp per window; a warp takes WINDOWS_PER_TASK consecutive windows
// and walks the sequences they belong to.  EMIT = build pairs, else the
// debug sketch export.  Five resident blocks per SM (48 registers).
template <int R, int KC, bool EMIT>
__global__ void __launch_bounds__(BT, 5) k_sketch(SketchParams p, uint32_t n_seq, const uint8_t* __restrict__ seq,
                                               const uint64_t* __restrict__ offs,
                                               const uint64_t* __restrict__ win_offs, uint64_t n_windows,
                                               uint32_t gw_base, uint64_t* __restrict__ pairs,
                                               uint32_t* __restrict__ sketch, uint32_t* __restrict__ counts,
                                               unsigned long long* real_pairs) {
    __shared__ uint32_t cand_sm[NWARP][SK_NW * 32];
    const uint32_t lane = lane_id();
    uint32_t* cand = cand_sm[threadIdx.x >> 5];
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t n_tasks = (n_windows + WINDOWS_PER_TASK - 1) / WINDOWS_PER_TASK;
    unsigned long long real = 0;
    for (uint64_t task = warp; task < n_tasks; task += n_warps) {
        uint64_t w0 = task * WINDOWS_PER_TASK;
        uint64_t w1 = min(w0 + WINDOWS_PER_TASK, n_windows);
        // sequence of w0: last i with win_offs[i] <= w0
        uint32_t lo = 0, hi = n_seq;  // invariant: win_offs[lo] <= w0 < win_offs[hi]
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (win_offs[mid] <= w0) lo = mid; else hi = mid;
        }
        uint32_t t = lo;
        for (uint64_t lw = w0; lw < w1; lw += SK_NW) {
            const uint8_t* sq[SK_NW];
            uint64_t Ls[SK_NW], wss[SK_NW];
            bool act[SK_NW];
#pragma unroll
            for (int i = 0; i < SK_NW; ++i) {
                const uint64_t x = lw + i;
                act[i] = x < w1;
                if (act[i]) {
                    while (win_offs[t + 1] <= x) ++t;
                    sq[i] = seq + offs[t];
                    Ls[i] = offs[t + 1] - offs[t];
                    wss[i] = (x - win_offs[t]) * p.stride;
                } else {
                    sq[i] = seq;
                    Ls[i] = 0;
                    wss[i] = 0;
                }
            }
            uint32_t f[SK_NW], cnt[SK_NW];
            warp_sketch_multi<R, SK_NW, KC>(sq, Ls, wss, act, p, cand, f, cnt);
#pragma unroll
            for (int i = 0; i < SK_NW; ++i) {
                if (!act[i]) continue;
                const uint64_t x = lw + i;
                if (EMIT) {
                    if (lane < p.s) {
                        uint64_t v = lane < cnt[i] ? (((uint64_t)hash_h2(f[i]) << 32) | (uint32_t)(gw_base + x))
                                                   : SENTINEL_PAIR;
                        pairs[x * p.s + lane] = v;
                    }
                    real += cnt[i];
                } else {
                    if (lane < p.s) sketch[x * p.s + lane] = lane < cnt[i] ? f[i] : 0u;
                    if (lane == 0) counts[x] = cnt[i];
                }
            }
        }
    }
    if (EMIT && lane == 0 && real) atomicAdd(real_pairs, real);
}

template <bool EMIT>
cudaError_t launch_sketch(const SketchParams& p, uint32_t n_seq, const uint8_t* seq, const uint64_t* offs,
                          const uint64_t* win_offs, uint64_t n_windows, uint32_t gw_base, uint64_t* pairs,
                          uint32_t* sketch, uint32_t* counts, unsigned long long* real, cudaStream_t s) {
    if (n_windows == 0) return cudaSuccess;
    uint64_t tasks = (n_windows + WINDOWS_PER_TASK - 1) / WINDOWS_PER_TASK;
    uint64_t blocks = (tasks + NWARP - 1) / NWARP;
    uint32_t g = grid_for(blocks, 16);
    const int r = sketch_r_for(p.w);
    const char* name = EMIT ? "sketch_emit" : "sketch";
#define MC_SK(RR, KK) \
    MC_LAUNCH(name, s, k_sketch<RR, KK, EMIT><<<g, BT, 0, s>>>(p, n_seq, seq, offs, win_offs, n_windows, gw_base, pairs, sketch, counts, real))
    if (r == 4) {
        if (p.k == 16) MC_SK(4, 16); else MC_SK(4, 0);
    } else if (r == 8) {
        if (p.k == 16) MC_SK(8, 16); else MC_SK(8, 0);
    } else {
        if (p.k == 16) MC_SK(16, 16); else MC_SK(16, 0);
    }
#undef MC_SK
    return cudaGetLastError();
}
}  // namespace

cudaError_t sketch_windows(const SketchParams& p, uint32_t n_seq, const uint8_t* seq, const uint64_t* offs,
                           const uint64_t* win_offs, uint64_t n_windows, uint32_t* sketch, uint32_t* counts,
                           cudaStream_t s) {
    return launch_sketch<false>(p, n_seq, seq, offs, win_offs, n_windows, 0, nullptr, sketch, counts, nullptr, s);
}

cudaError_t emit_pairs(const SketchParams& p, uint32_t n_targets, const uint8_t* seq, const uint64_t* offs,
                       const uint64_t* win_offs, uint64_t n_windows, uint32_t gw_base, uint64_t* pairs,
                       unsigned long long* real_pairs, cudaStream_t s) {
    return launch_sketch<true>(p, n_targets, seq, offs, win_offs, n_windows, gw_base, pairs, nullptr, nullptr,
                               real_pairs, s);
}

// ------------------------------------------------------------ radix sort
// Single-pass LSD radix sort (one kernel per 8-bit digit; Merrill and
// Garland's decoupled look-back, as in "Onesweep", Adinets and Merrill
// 2022).  One streaming read computes the digit totals of all four passes;
// then every pass reads each pair once and writes it once.  A tile
// (4,096 pairs) ranks its pairs by digit, publishes its per-digit counts,
// looks back over earlier tiles' published counts for its global offsets,
// and writes each digit's run with consecutive threads on consecutive
// addresses.
namespace {
constexpr int RS_ITEMS = 16;
constexpr uint64_t RS_TILE = (uint64_t)BT * RS_ITEMS;  // 4096 pairs
constexpr int RS_BLOCKS_PER_SM = 3;
constexpr int RS_LOOKBACK = 4;  // earlier tiles read per look-back step
// element of (warp w, round i, lane l) in a tile: w*32*RS_ITEMS + i*32 + l

// Look-back status word of (tile, digit): kind (2 bits: 1 = this tile's
// count, 2 = inclusive prefix over tiles 0..tile), pass tag (4 bits: pass +
// 1, so that one zeroing serves all four passes), value (58 bits).
constexpr uint64_t ST_COUNT = 1ull << 62;
constexpr uint64_t ST_PREFIX = 2ull << 62;
constexpr uint64_t ST_VALUE = (1ull << 58) - 1;
constexpr uint64_t LOOKBACK_LIMIT_NS = 2000000000ull;  // a wait longer than this is an error

__device__ __forceinline__ uint64_t ld_relaxed_gpu(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Digit totals of the four passes (sentinels excluded): totals[pass][digit].
__global__ void __launch_bounds__(BT) k_radix_totals(const uint64_t* __restrict__ in, uint64_t n,
                                                     unsigned long long* __restrict__ totals) {
    __shared__ uint32_t sh[NWARP][4][256];
    for (int i = threadIdx.x; i < NWARP * 1024; i += BT) (&sh[0][0][0])[i] = 0;
    __syncthreads();
    const int w = threadIdx.x >> 5;
    const uint64_t stride = (uint64_t)gridDim.x * BT * 4;
    for (uint64_t e0 = (uint64_t)blockIdx.x * BT * 4 + threadIdx.x; e0 < n; e0 += stride) {
        uint64_t v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const uint64_t e = e0 + (uint64_t)i * BT;
            v[i] = e < n ? in[e] : SENTINEL_PAIR;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (v[i] == SENTINEL_PAIR) continue;
            const uint32_t k = (uint32_t)(v[i] >> 32);
            atomicAdd(&sh[w][0][k & 255u], 1u);
            atomicAdd(&sh[w][1][(k >> 8) & 255u], 1u);
            atomicAdd(&sh[w][2][(k >> 16) & 255u], 1u);
            atomicAdd(&sh[w][3][k >> 24], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 1024; i += BT) {
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < NWARP; ++j) c += (&sh[j][0][0])[i];
        if (c) atomicAdd(totals + i, (unsigned long long)c);
    }
}

// Rank of round i of a warp's 32 pairs: the lanes holding the same digit
// (each lane sets its bit in the digit's word of a per-warp mask table in
// shared memory, then reads the word back; two tables alternate so that a
// table's reset is ordered before its next use by the warp barriers of the
// round in between) and the warp's running count of that digit.  Invalid
// lanes carry digit 256, which is neither counted nor reset.
__device__ __forceinline__ uint32_t rank_round(int i, bool valid, uint32_t d, uint32_t lane, uint32_t lt,
                                               uint32_t* wcount, uint32_t* mask0, uint32_t* mask1) {
    uint32_t* mask = (i & 1) ? mask1 : mask0;
    atomicOr(&mask[d], 1u << lane);
    __syncwarp();
    const uint32_t peers = mask[d];
    __syncwarp();
    const uint32_t rank = __popc(peers & lt);
    const uint32_t leader = (__ffs(peers) - 1) & 31u;
    uint32_t before = 0;
    if (valid && rank == 0) {
        before = atomicAdd(&wcount[d], (uint32_t)__popc(peers));
        mask[d] = 0;
    }
    return __shfl_sync(FULL_MASK, before, leader) + rank;
}

// One pass over digit `pass` (bits 32 + 8 pass ..).  Persistent blocks take
// tiles in order from *tile_ctr, so a tile only ever waits for tiles that
// running blocks hold.  FILTER drops sentinel pairs (first pass).
template <bool FILTER>
__global__ void __launch_bounds__(BT, RS_BLOCKS_PER_SM)
    k_radix_pass(const uint64_t* __restrict__ in, uint64_t* __restrict__ out, uint64_t n, uint32_t pass,
                 const unsigned long long* __restrict__ totals, uint64_t* status, uint32_t* tile_ctr,
                 uint64_t n_tiles, uint64_t limit_ns, uint32_t* err) {
    __shared__ uint32_t wc[NWARP][257];       // per-warp digit counts, then tile offsets
    __shared__ uint32_t peer_mask[2][NWARP][257];
    __shared__ uint64_t gdelta[256];          // global position of a digit's run minus its tile offset
    __shared__ uint64_t staged[RS_TILE];
    __shared__ uint64_t sm[NWARP];
    __shared__ uint32_t s_tile;
    const int w = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    const uint32_t sel = 0x4440u + pass;  // __byte_perm selector of byte `pass` of the key
    const uint64_t tag = (uint64_t)(pass + 1) << 58;
    for (int i = threadIdx.x; i < 2 * NWARP * 257; i += BT) (&peer_mask[0][0][0])[i] = 0;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
    uint64_t all;
    const uint64_t dbase = block_exclusive((uint64_t)totals[threadIdx.x], (uint64_t)0, OpSum(), sm, &all);
    uint64_t tile = s_tile;
    while (tile < n_tiles) {
        for (int i = threadIdx.x; i < NWARP * 257; i += BT) (&wc[0][0])[i] = 0;
        __syncthreads();
        uint64_t v[RS_ITEMS];
        uint32_t dr[RS_ITEMS];  // digit << 16 | rank within the warp's pairs of that digit
        const uint64_t base = tile * RS_TILE + (uint64_t)w * 32 * RS_ITEMS + lane;
        if ((tile + 1) * RS_TILE <= n) {
#pragma unroll
            for (int i = 0; i < RS_ITEMS; ++i) v[i] = in[base + (uint64_t)i * 32];
#pragma unroll
            for (int i = 0; i < RS_ITEMS; ++i) {
                const bool valid = !FILTER || v[i] != SENTINEL_PAIR;
                const uint32_t d = valid ? __byte_perm((uint32_t)(v[i] >> 32), 0, sel) : 256u;
                dr[i] = (d << 16) | rank_round(i, valid, d, lane, lt, wc[w], peer_mask[0][w], peer_mask[1][w]);
            }
        } else {
#pragma unroll
            for (int i = 0; i < RS_ITEMS; ++i) {
                const uint64_t e = base + (uint64_t)i * 32;
                v[i] = e < n ? in[e] : SENTINEL_PAIR;
            }
#pragma unroll
            for (int i = 0; i < RS_ITEMS; ++i) {
                const bool valid = base + (uint64_t)i * 32 < n && (!FILTER || v[i] != SENTINEL_PAIR);
                const uint32_t d = valid ? __byte_perm((uint32_t)(v[i] >> 32), 0, sel) : 256u;
                dr[i] = (d << 16) | rank_round(i, valid, d, lane, lt, wc[w], peer_mask[0][w], peer_mask[1][w]);
            }
        }
        __syncthreads();
        // thread d: exclusive offsets of digit d over the warps, tile count
        uint32_t run = 0;
#pragma unroll
        for (int i = 0; i < NWARP; ++i) {
            const uint32_t c = wc[i][threadIdx.x];
            wc[i][threadIdx.x] = run;
            run += c;
        }
        // publish, then look back for the count of digit d in earlier tiles
        uint64_t excl = 0;
        uint64_t* mine = status + tile * 256 + threadIdx.x;
        if (tile == 0) {
            st_relaxed_gpu(mine, ST_PREFIX | tag | run);
        } else {
            st_relaxed_gpu(mine, ST_COUNT | tag | run);
            int64_t t = (int64_t)tile - 1;
            uint64_t t0 = 0;
            uint32_t polls = 0;
            while (true) {
                uint64_t st[RS_LOOKBACK];
#pragma unroll
                for (int k = 0; k < RS_LOOKBACK; ++k)
                    st[k] = t - k >= 0 ? ld_relaxed_gpu(status + (uint64_t)(t - k) * 256 + threadIdx.x)
                                       : ST_PREFIX | tag;
                uint32_t used = 0;
                bool stop = false, done = false;
#pragma unroll
                for (int k = 0; k < RS_LOOKBACK; ++k) {
                    if (!stop) {
                        if ((st[k] & (15ull << 58)) != tag || (st[k] >> 62) == 0) {
                            stop = true;  // not published in this pass yet
                        } else {
                            excl += st[k] & ST_VALUE;
                            ++used;
                            if ((st[k] >> 62) == 2) stop = done = true;
                        }
                    }
                }
                if (done) break;
                t -= used;
                if (used == 0 && (++polls & 255u) == 0) {
                    const uint64_t now = globaltimer_ns();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > limit_ns) {
                        atomicMax(err, 1u);
                        break;
                    }
                }
            }
            st_relaxed_gpu(mine, ST_PREFIX | tag | (excl + run));
        }
        uint64_t tot;
        const uint32_t ds = (uint32_t)block_exclusive((uint64_t)run, (uint64_t)0, OpSum(), sm, &tot);
        gdelta[threadIdx.x] = dbase + excl - ds;
#pragma unroll
        for (int i = 0; i < NWARP; ++i) wc[i][threadIdx.x] += ds;
        __syncthreads();
        // stage in digit order, then write each digit's run
#pragma unroll
        for (int i = 0; i < RS_ITEMS; ++i) {
            const uint32_t d = dr[i] >> 16;
            if (d < 256u) staged[wc[w][d] + (dr[i] & 0xFFFFu)] = v[i];
        }
        __syncthreads();
        const uint32_t count = (uint32_t)tot;
        for (uint32_t j = threadIdx.x; j < count; j += BT) {
            const uint64_t x = staged[j];
            out[gdelta[__byte_perm((uint32_t)(x >> 32), 0, sel)] + j] = x;
        }
        if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
        __syncthreads();
        tile = s_tile;
    }
}
// One-shot stall of the next sort's last pass (mc_debug_stall_next_sort):
// the wait limit of that pass in ns, 0 = not armed.
std::atomic<uint64_t> g_stall_limit_ns{0};
}  // namespace

void arm_sort_stall(uint64_t limit_ns) { g_stall_limit_ns.store(limit_ns); }

cudaError_t sort_pairs(const Mem& mem, uint64_t* a, uint64_t* b, uint64_t n_total, uint64_t n_real, cudaStream_t s) {
    if (n_total == 0) return cudaSuccess;
    // An armed stall makes the last pass start at tile 1: tile 0's counts are
    // never published, so tile 1's look-back wait gives up after the armed
    // limit.  Every look-back sum stays a sum over a subset of earlier tiles'
    // counts, so every write stays inside the pass's output; only the last
    // pass is disturbed, because an earlier one would hand the next pass
    // data whose digits disagree with the digit totals.
    const uint64_t stall_ns = g_stall_limit_ns.exchange(0);
    const uint64_t max_tiles = (n_total + RS_TILE - 1) / RS_TILE;
    // control block: totals[4][256], tile counters[4], error word
    constexpr size_t CTRL_WORDS = 4 * 256 + 3;
    Tmp<uint64_t> ctrl(mem, CTRL_WORDS, s);
    Tmp<uint64_t> status(mem, max_tiles * 256, s);
    if (!ctrl.ok() || !status.ok()) return cudaErrorMemoryAllocation;
    unsigned long long* totals = (unsigned long long*)ctrl.ptr;
    uint32_t* tile_ctr = (uint32_t*)(ctrl.ptr + 4 * 256);
    uint32_t* err = tile_ctr + 4;
    cudaError_t e = cudaMemsetAsync(ctrl.ptr, 0, CTRL_WORDS * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status.ptr, 0, max_tiles * 256 * 8, s);
    if (e != cudaSuccess) return e;
    MC_LAUNCH("radix_totals", s,
              k_radix_totals<<<grid_for((n_total + 4 * BT - 1) / (4 * BT), 4), BT, 0, s>>>(a, n_total, totals));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    uint64_t* src = a;
    uint64_t* dst = b;
    for (uint32_t pass = 0; pass < 4; ++pass) {
        const uint64_t n = pass == 0 ? n_total : n_real;
        if (n == 0) break;
        const uint64_t tiles = (n + RS_TILE - 1) / RS_TILE;
        const uint32_t g = grid_for(tiles, RS_BLOCKS_PER_SM);
        const unsigned long long* tp = totals + 256 * pass;
        uint64_t limit = LOOKBACK_LIMIT_NS;
        if (stall_ns && pass == 3 && tiles >= 2) {
            limit = stall_ns;
            e = cudaMemsetAsync(tile_ctr + pass, 1, 1, s);  // the counter's low byte: tiles are taken from 1
            if (e != cudaSuccess) return e;
        }
        if (pass == 0)
            MC_LAUNCH("radix_pass", s,
                      k_radix_pass<true><<<g, BT, 0, s>>>(src, dst, n, pass, tp, status.ptr, tile_ctr + pass, tiles,
                                                          limit, err));
        else
            MC_LAUNCH("radix_pass", s,
                      k_radix_pass<false><<<g, BT, 0, s>>>(src, dst, n, pass, tp, status.ptr, tile_ctr + pass, tiles,
                                                           limit, err));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint64_t* t = src;
        src = dst;
        dst = t;
    }
    // after 4 passes the data is back in `a`; a look-back that gave up
    // leaves a wrong order, which is reported as a timeout
    uint32_t h_err = 0;
    e = cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    return h_err ? cudaErrorTimeout : cudaSuccess;
}

// --------------------------------------------------------------- finalize
namespace {
constexpr int FIN_ITEMS = 8;
constexpr uint64_t FIN_TILE = (uint64_t)BT * FIN_ITEMS;  // warp w: [base + 256 w, base + 256 (w+1))
constexpr uint32_t FIN_BUCKETS = 4096;  // window ranges of the target lookup table
constexpr uint32_t FIN_WB_SMEM_MAX = 12288;  // window bases k_fin_emit keeps in shared memory (48 KiB)

__device__ __forceinline__ uint32_t hk_of(uint64_t v) { return (uint32_t)(v >> 32); }

// In the sorted pair array, e starts a feature's run if its predecessor has
// another feature; e is kept (rank in its run < cap) unless the pair cap
// places earlier has the same feature (runs are contiguous).  Sentinel
// pairs may end a run (the part a sharded build gives up to earlier
// shards, finalize_after): they are neither kept nor starts, and a pair
// after one starts a new run.
__device__ __forceinline__ bool same_feature(uint64_t x, uint32_t hk) {
    return x != SENTINEL_PAIR && hk_of(x) == hk;
}

// The pair, its predecessor and the pair cap places earlier are loaded
// together (each only bounded by the array), so that the loads of all the
// items a thread handles are in flight at once.
__device__ __forceinline__ void fin_flags(const uint64_t* __restrict__ a, uint64_t n, uint32_t cap, uint64_t e,
                                          uint64_t& v, bool& st, bool& kept, bool& over) {
    st = kept = over = false;
    const bool in = e < n;
    v = in ? a[e] : SENTINEL_PAIR;
    const uint64_t prev = (in && e > 0) ? a[e - 1] : SENTINEL_PAIR;
    const uint64_t back = (in && e >= cap) ? a[e - cap] : SENTINEL_PAIR;
    if (!in || v == SENTINEL_PAIR) return;
    const uint32_t hk = hk_of(v);
    st = e == 0 || !same_feature(prev, hk);
    const bool dropped = e >= cap && same_feature(back, hk);
    kept = !dropped;
    // the first dropped pair of an overflowing run: the pair cap earlier starts the run
    over = dropped && (e == cap || !same_feature(a[e - cap - 1], hk));
}

// Tile sums of kept pairs and run starts.
__global__ void __launch_bounds__(BT) k_fin_count(const uint64_t* __restrict__ a, uint64_t n, uint32_t cap,
                                                  uint64_t* __restrict__ tkept, uint64_t* __restrict__ tkeys,
                                                  uint64_t n_tiles) {
    __shared__ uint64_t sm[NWARP];
    const int w = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint64_t base = tile * FIN_TILE + (uint64_t)w * 32 * FIN_ITEMS + lane;
        uint32_t nk = 0, ns = 0;
#pragma unroll
        for (int i = 0; i < FIN_ITEMS; ++i) {
            uint64_t v;
            bool st, kept, over;
            fin_flags(a, n, cap, base + (uint64_t)i * 32, v, st, kept, over);
            nk += kept;
            ns += st;
        }
        const uint64_t both = block_reduce(((uint64_t)ns << 32) | nk, (uint64_t)0, OpSum(), sm);
        if (threadIdx.x == 0) {
            tkept[tile] = both & 0xFFFFFFFFull;
            tkeys[tile] = both >> 32;
        }
    }
}

// Writes the condensed outputs at the scanned positions: locations of kept
// pairs (global window -> (target, window), 32-bit target << jbits | window
// when jbits > 0, else 64-bit target << 32 | window), and per feature its h2 value,
// the position of its first location and the index of its first pair.
// The target of a global window gw is the last t with wbase[t] <= gw; a
// block first tabulates that target for the first window of each of
// FIN_BUCKETS equal window ranges, which narrows every search to the
// targets that overlap gw's range (one or two for genome-sized targets).
// With wb_smem, wbase (n_targets + 1 words) is copied to shared memory too,
// so that the search and the window offset are shared-memory reads.
__global__ void __launch_bounds__(BT) k_fin_emit(const uint64_t* __restrict__ a, uint64_t n, uint32_t cap,
                                                 const uint64_t* __restrict__ tkept, const uint64_t* __restrict__ tkeys,
                                                 uint64_t n_tiles, const uint32_t* __restrict__ wbase,
                                                 uint32_t n_targets, uint32_t jbits, void* __restrict__ locs,
                                                 uint32_t* __restrict__ khk, uint64_t* __restrict__ koff,
                                                 uint64_t* __restrict__ kstart, unsigned long long* overflow,
                                                 bool wb_smem) {
    extern __shared__ uint32_t fin_smem[];
    uint32_t* first_target = fin_smem;  // FIN_BUCKETS + 1 words
    __shared__ uint32_t wk[NWARP], wsx[NWARP];
    const int w = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    const uint32_t* wb = wbase;
    if (wb_smem) {
        uint32_t* copy = fin_smem + FIN_BUCKETS + 1;
        for (uint32_t t = threadIdx.x; t <= n_targets; t += BT) copy[t] = wbase[t];
        __syncthreads();
        wb = copy;
    }
    const uint64_t n_win = wb[n_targets];
    uint32_t bshift = 0;
    while ((n_win >> bshift) >= FIN_BUCKETS) ++bshift;
    for (uint32_t b = threadIdx.x; b <= FIN_BUCKETS; b += BT) {
        const uint64_t x = (uint64_t)b << bshift;
        uint32_t lo = 0, hi = n_targets;  // last t with wb[t] <= x
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (wb[mid] <= x) lo = mid; else hi = mid;
        }
        first_target[b] = lo;
    }
    __syncthreads();
    unsigned long long n_over = 0;
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint64_t base = tile * FIN_TILE + (uint64_t)w * 32 * FIN_ITEMS + lane;
        uint64_t v[FIN_ITEMS];
        uint32_t kmask = 0, smask = 0;  // per item: kept / run start
        uint32_t nk = 0, ns = 0;
#pragma unroll
        for (int i = 0; i < FIN_ITEMS; ++i) {
            bool st, kept, over;
            fin_flags(a, n, cap, base + (uint64_t)i * 32, v[i], st, kept, over);
            kmask |= (kept ? 1u : 0u) << i;
            smask |= (st ? 1u : 0u) << i;
            nk += __popc(__ballot_sync(FULL_MASK, kept));
            ns += __popc(__ballot_sync(FULL_MASK, st));
            n_over += over;
        }
        if (lane == 0) {
            wk[w] = nk;
            wsx[w] = ns;
        }
        __syncthreads();
        uint64_t kpos = tkept[tile], kidx = tkeys[tile];
        for (int i = 0; i < w; ++i) {
            kpos += wk[i];
            kidx += wsx[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < FIN_ITEMS; ++i) {
            const bool kept = (kmask >> i) & 1u, st = (smask >> i) & 1u;
            const uint32_t bk = __ballot_sync(FULL_MASK, kept);
            const uint32_t bs = __ballot_sync(FULL_MASK, st);
            const uint64_t my_k = kpos + __popc(bk & lt);
            if (kept) {
                const uint32_t gw = (uint32_t)v[i];
                const uint32_t rng = gw >> bshift;  // < FIN_BUCKETS since gw < n_win
                uint32_t lo = first_target[rng];    // last t with wb[t] <= gw lies in [lo, hi)
                uint32_t hi = min(first_target[rng + 1] + 1, n_targets);
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (wb[mid] <= gw) lo = mid; else hi = mid;
                }
                if (jbits)
                    static_cast<uint32_t*>(locs)[my_k] = (lo << jbits) | (gw - wb[lo]);
                else
                    static_cast<uint64_t*>(locs)[my_k] = ((uint64_t)lo << 32) | (gw - wb[lo]);
            }
            if (st) {
                const uint64_t my_s = kidx + __popc(bs & lt);
                khk[my_s] = hk_of(v[i]);
                koff[my_s] = my_k;
                kstart[my_s] = base + (uint64_t)i * 32;
            }
            kpos += __popc(bk);
            kidx += __popc(bs);
        }
    }
    for (int o = 16; o >= 1; o >>= 1) n_over += __shfl_xor_sync(FULL_MASK, n_over, o);
    if (lane == 0 && n_over) atomicAdd(overflow, n_over);
}

// Pairs (h2 << 32 | global window) of a finalized layout, in layout order:
// the input of the next finalize after an extension.
__global__ void k_reconstruct_pairs(const uint64_t* __restrict__ table, uint64_t table_len, TableFmt fmt,
                                    const void* __restrict__ locs, uint32_t jbits,
                                    const uint32_t* __restrict__ wbase, uint64_t* __restrict__ out) {
    const uint32_t jmask = jbits ? (1u << jbits) - 1u : 0u;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < table_len;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t e = table[i];
        if (e == 0) continue;
        const uint64_t off = fmt.offset(e);
        const uint32_t cnt = fmt.count(e);
        const uint64_t hk = (uint64_t)fmt.key(e, i) << 32;
        for (uint32_t j = 0; j < cnt; ++j) {
            uint32_t t, w;
            if (jbits) {
                const uint32_t x = static_cast<const uint32_t*>(locs)[off + j];
                t = x >> jbits;
                w = x & jmask;
            } else {
                const uint64_t x = static_cast<const uint64_t*>(locs)[off + j];
                t = (uint32_t)(x >> 32);
                w = (uint32_t)x;
            }
            out[off + j] = hk | (uint32_t)(wbase[t] + w);
        }
    }
}

// Exclusive max-scan of the tile maxima (one block; the tiles are few).
__global__ void __launch_bounds__(BT) k_exclusive_max_i64(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                                          uint64_t n, int64_t* total) {
    __shared__ int64_t sm[NWARP];
    int64_t carry = INT64_MIN;
    for (uint64_t base = 0; base < n; base += BT) {
        uint64_t e = base + threadIdx.x;
        int64_t v = e < n ? in[e] : INT64_MIN;
        int64_t tot;
        int64_t ex = block_exclusive(v, (int64_t)INT64_MIN, OpMaxI(), sm, &tot);
        if (e < n) out[e] = max(carry, ex);
        carry = max(carry, tot);
    }
    if (threadIdx.x == 0) *total = carry;
}

__device__ __forceinline__ uint64_t home_slot(uint32_t hk, uint32_t log_t) {
    return log_t >= 32 ? hk : (hk >> (32 - log_t));
}

// Tile maxima of home(k) - k.
__global__ void __launch_bounds__(BT) k_tab_dispmax(const uint32_t* __restrict__ khk, uint64_t n, uint32_t log_t,
                                                    int64_t* __restrict__ tmax, uint64_t n_tiles) {
    __shared__ int64_t sm[NWARP];
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        uint64_t base = tile * FIN_TILE;
        int64_t m = INT64_MIN;
#pragma unroll
        for (int i = 0; i < FIN_ITEMS; ++i) {
            uint64_t e = base + (uint64_t)i * BT + threadIdx.x;
            if (e < n) m = max(m, (int64_t)home_slot(khk[e], log_t) - (int64_t)e);
        }
        int64_t tot = block_reduce(m, (int64_t)INT64_MIN, OpMaxI(), sm);
        if (threadIdx.x == 0) tmax[tile] = tot;
    }
}

// slot(k) = k + max(prefix, inclusive max of home - k); writes the packed
// word (count = kept locations, koff[k + 1] - koff[k]).  A displacement beyond the word's field sets *too_far (the host then
// retries with a larger table).
__global__ void __launch_bounds__(BT) k_tab_emit(const uint32_t* __restrict__ khk, const uint64_t* __restrict__ koff,
                                                 uint64_t n, TableFmt fmt, const int64_t* __restrict__ tpre, uint64_t n_tiles,
                                                 uint64_t* __restrict__ table, unsigned int* max_disp,
                                                 unsigned int* too_far) {
    __shared__ int64_t sm[NWARP];
    __shared__ uint64_t smu[NWARP];
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        uint64_t base = tile * FIN_TILE;
        int64_t carry = tpre[tile];
        uint64_t dmax = 0;
        for (int i = 0; i < FIN_ITEMS; ++i) {
            uint64_t e = base + (uint64_t)i * BT + threadIdx.x;
            bool in_range = e < n;
            uint32_t hk = in_range ? khk[e] : 0;
            uint64_t home = fmt.home(hk);
            int64_t a = in_range ? (int64_t)home - (int64_t)e : INT64_MIN;
            int64_t tot;
            int64_t ex = block_exclusive(a, (int64_t)INT64_MIN, OpMaxI(), sm, &tot);
            int64_t inc = max(carry, max(ex, a));
            carry = max(carry, tot);
            if (in_range) {
                uint64_t slot = (uint64_t)((int64_t)e + inc);
                const uint32_t cnt = (uint32_t)(koff[e + 1] - koff[e]);  // kept locations (<= cap)
                const uint64_t disp = slot - home;
                if (disp > TAB_MAX_DISP) atomicMax(too_far, 1u);
                table[slot] = fmt.pack(koff[e], hk, (uint32_t)(disp & TAB_MAX_DISP), cnt);
                dmax = max(dmax, disp);
            }
        }
        uint64_t dm = block_reduce(dmax, (uint64_t)0, OpMaxU(), smu);
        if (threadIdx.x == 0) atomicMax(max_disp, (unsigned int)min(dm, (uint64_t)0xFFFFFFFFu));
    }
}
}  // namespace

cudaError_t reconstruct_pairs(const uint64_t* table, uint64_t table_len, TableFmt fmt, const void* locs, uint32_t jbits,
                              const uint32_t* wbase, uint64_t* out, cudaStream_t s) {
    if (table_len == 0) return cudaSuccess;
    MC_LAUNCH("reconstruct_pairs", s,
              k_reconstruct_pairs<<<grid_for((table_len + BT - 1) / BT), BT, 0, s>>>(table, table_len, fmt, locs, jbits,
                                                                                     wbase, out));
    return cudaGetLastError();
}

cudaError_t finalize_pairs(const Mem& mem, const uint64_t* sorted, uint64_t n, uint32_t cap, const uint32_t* wbase,
                           uint32_t n_targets, uint32_t jbits, FinalizeOut* out, cudaStream_t s) {
    cudaError_t e;
    *out = FinalizeOut();
    const uint64_t tiles = (n + FIN_TILE - 1) / FIN_TILE;
    const uint32_t g = grid_for(tiles ? tiles : 1);
    // counters: [0] overflow keys, [1] max displacement (u32 in low word),
    // [2] displacement beyond the word's field
    Tmp<unsigned long long> ctr(mem, 4, s);
    if (!ctr.ok()) return cudaErrorMemoryAllocation;
    if ((e = cudaMemsetAsync(ctr.ptr, 0, 4 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
    uint64_t host_tot[2] = {0, 0};
    Tmp<uint64_t> tkept(mem, tiles + 1, s), tkeys(mem, tiles + 1, s);
    if (!tkept.ok() || !tkeys.ok()) return cudaErrorMemoryAllocation;
    if (n > 0) {
        MC_LAUNCH("fin_count", s, k_fin_count<<<g, BT, 0, s>>>(sorted, n, cap, tkept.ptr, tkeys.ptr, tiles));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = scan_exclusive_sum(mem, tkept.ptr, tkept.ptr, tiles, s)) != cudaSuccess) return e;
        if ((e = scan_exclusive_sum(mem, tkeys.ptr, tkeys.ptr, tiles, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&host_tot[0], tkept.ptr + tiles, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(&host_tot[1], tkeys.ptr + tiles, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    }
    const uint64_t n_kept = host_tot[0], n_keys = host_tot[1];
    // table format: slots = 2^log_t >= 2 n_keys (load factor <= 1/2), and
    // enough offset bits for every location; a larger table is taken when
    // a displacement does not fit the word's field
    TableFmt fmt{1, count_bits(cap)};
    while ((1ull << fmt.log_t) < 2 * n_keys) ++fmt.log_t;
    while (fmt.log_t <= 32 && fmt.obits() < 64 && (n_kept >> fmt.obits()) != 0) ++fmt.log_t;
    if (fmt.log_t > 32) {
        out->table_full = true;
        return cudaSuccess;
    }
    Tmp<unsigned char> locs(mem, n_kept * loc_bytes(jbits), s);
    Tmp<uint64_t> koff(mem, n_keys + 1, s), kstart(mem, n_keys + 1, s);
    Tmp<uint32_t> khk(mem, n_keys, s);
    if (!locs.ok() || !koff.ok() || !kstart.ok() || !khk.ok()) return cudaErrorMemoryAllocation;
    if (n > 0) {
        // wbase in shared memory when it fits next to the range table
        const bool wb_smem = n_targets + 1 <= FIN_WB_SMEM_MAX;
        const size_t smem = (size_t)(FIN_BUCKETS + 1 + (wb_smem ? n_targets + 1 : 0)) * 4;
        if ((e = cudaFuncSetAttribute(k_fin_emit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        MC_LAUNCH("fin_emit", s,
                  k_fin_emit<<<g, BT, smem, s>>>(sorted, n, cap, tkept.ptr, tkeys.ptr, tiles, wbase, n_targets, jbits,
                                                 locs.ptr, khk.ptr, koff.ptr, kstart.ptr, ctr.ptr, wb_smem));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(kstart.ptr + n_keys, &n, 8, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(koff.ptr + n_keys, &n_kept, 8, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    }
    const uint64_t ktiles = (n_keys + FIN_TILE - 1) / FIN_TILE;
    Tmp<int64_t> kt_max(mem, ktiles + 1, s), kt_pre(mem, ktiles + 1, s);
    if (!kt_max.ok() || !kt_pre.ok()) return cudaErrorMemoryAllocation;
    unsigned long long host_ctr[3] = {0, 0, 0};
    for (;;) {
        const uint64_t T = 1ull << fmt.log_t;
        int64_t host_maxa = INT64_MIN;
        if (n_keys > 0) {
            MC_LAUNCH("tab_dispmax", s,
                      k_tab_dispmax<<<grid_for(ktiles), BT, 0, s>>>(khk.ptr, n_keys, fmt.log_t, kt_max.ptr, ktiles));
            MC_LAUNCH("exclusive_max_i64", s,
                      k_exclusive_max_i64<<<1, BT, 0, s>>>(kt_max.ptr, kt_pre.ptr, ktiles, kt_pre.ptr + ktiles));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = cudaMemcpyAsync(&host_maxa, kt_pre.ptr + ktiles, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        }
        const uint64_t last_slot = n_keys ? (uint64_t)((int64_t)(n_keys - 1) + host_maxa) : 0;
        // two empty words past the last key or the home slots, rounded to whole 32-byte sectors
        const uint64_t table_len = (((last_slot + 1 > T ? last_slot + 1 : T) + 2) + 3) & ~3ull;
        Tmp<uint64_t> table(mem, table_len, s);
        if (!table.ok()) return cudaErrorMemoryAllocation;
        if ((e = cudaMemsetAsync(table.ptr, 0, table_len * sizeof(uint64_t), s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(ctr.ptr + 1, 0, 2 * sizeof(unsigned long long), s)) != cudaSuccess) return e;
        if (n_keys > 0) {
            MC_LAUNCH("tab_emit", s,
                      k_tab_emit<<<grid_for(ktiles), BT, 0, s>>>(khk.ptr, koff.ptr, n_keys, fmt, kt_pre.ptr, ktiles,
                                                                 table.ptr,
                                                                 (unsigned int*)(ctr.ptr + 1),
                                                                 (unsigned int*)(ctr.ptr + 2)));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if ((e = cudaMemcpyAsync(host_ctr, ctr.ptr, 24, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if (host_ctr[2]) {  // a displacement beyond the word's field: twice the slots
            if (++fmt.log_t > 32) {
                out->table_full = true;
                return cudaSuccess;
            }
            continue;
        }
        out->table_len = table_len;
        out->table_bytes = table_len * sizeof(uint64_t);
        out->table = table.release();
        break;
    }
    out->n_keys = n_keys;
    out->n_kept = n_kept;
    out->overflow_keys = host_ctr[0];
    out->max_probe = (uint32_t)(host_ctr[1] & 0xFFFFFFFFull);
    out->fmt = fmt;
    out->locs = locs.release();
    return cudaSuccess;
}

// ------------------------------------------------------------ merge path
// Live extension (Section 4.1: new targets get the next ids): the stored
// pairs (reconstructed in layout order) and the sorted pairs of the new
// targets are two sorted runs; merging them gives the sorted pairs of the
// whole database without sorting the stored ones again.  Merge path
// (Odeh, Green, Mwassi, Shmueli, Birk 2012): a block takes 2,048
// consecutive outputs, finds where that output range starts and ends in
// both inputs by a binary search along the diagonals, stages the two input
// slices in shared memory, and each thread merges eight outputs.
namespace {
constexpr int MP_ITEMS = 8;
constexpr uint64_t MP_TILE = (uint64_t)BT * MP_ITEMS;

// Number of elements of a in the first d outputs of merge(a, b), ties
// taken from a first.
__device__ __forceinline__ uint64_t merge_split(const uint64_t* a, uint64_t na, const uint64_t* b, uint64_t nb,
                                                uint64_t d) {
    uint64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (a[mid] <= b[d - mid - 1]) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(BT) k_merge_path(const uint64_t* __restrict__ a, uint64_t na,
                                                   const uint64_t* __restrict__ b, uint64_t nb,
                                                   uint64_t* __restrict__ c) {
    __shared__ uint64_t in[MP_TILE];
    __shared__ uint64_t out[MP_TILE];
    __shared__ uint64_t split[2];
    const uint64_t n = na + nb;
    for (uint64_t d0 = (uint64_t)blockIdx.x * MP_TILE; d0 < n; d0 += (uint64_t)gridDim.x * MP_TILE) {
        const uint64_t d1 = min(d0 + MP_TILE, n);
        if (threadIdx.x < 2) split[threadIdx.x] = merge_split(a, na, b, nb, threadIdx.x ? d1 : d0);
        __syncthreads();
        const uint64_t i0 = split[0], i1 = split[1];
        const uint32_t ta = (uint32_t)(i1 - i0), tb = (uint32_t)((d1 - d0) - ta);
        for (uint32_t k = threadIdx.x; k < ta + tb; k += BT) in[k] = k < ta ? a[i0 + k] : b[(d0 - i0) + (k - ta)];
        __syncthreads();
        const uint64_t* sa = in;
        const uint64_t* sb = in + ta;
        const uint32_t dl = threadIdx.x * MP_ITEMS;
        if (dl < ta + tb) {
            uint32_t lo = dl > tb ? dl - tb : 0, hi = dl < ta ? dl : ta;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (sa[mid] <= sb[dl - mid - 1]) lo = mid + 1; else hi = mid;
            }
            uint32_t ia = lo, ib = dl - lo;
            for (uint32_t k = 0; k < MP_ITEMS && dl + k < ta + tb; ++k) {
                const bool take_a = ib >= tb || (ia < ta && sa[ia] <= sb[ib]);
                out[dl + k] = take_a ? sa[ia++] : sb[ib++];
            }
        }
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < ta + tb; k += BT) c[d0 + k] = out[k];
        __syncthreads();
    }
}
}  // namespace

cudaError_t merge_sorted_pairs(const uint64_t* a, uint64_t na, const uint64_t* b, uint64_t nb, uint64_t* c,
                               cudaStream_t s) {
    const uint64_t n = na + nb;
    if (n == 0) return cudaSuccess;
    MC_LAUNCH("merge_path", s,
              k_merge_path<<<grid_for((n + MP_TILE - 1) / MP_TILE, 4), BT, 0, s>>>(a, na, b, nb, c));
    return cudaGetLastError();
}

// ------------------------------------------------------- sharded builds
// Section 4.3 partitions the reference targets over GPUs.  A shard holds a
// contiguous range of target ids, so every location of an earlier shard is
// smaller than every location of a later one, and the cap smallest
// locations of a feature over all shards are: those of the earlier shards
// first.  A shard therefore keeps at most cap - prior(f) of its own
// locations of feature f, prior(f) = f's locations in the earlier shards
// (clamped to cap), and the union of the shards equals the database of all
// targets.
namespace {

// Run starts of sorted pairs: keys and start indices at the scanned
// positions tkeys (exclusive prefix of each tile's run starts).
__global__ void __launch_bounds__(BT) k_run_emit(const uint64_t* __restrict__ a, uint64_t n,
                                                 const uint64_t* __restrict__ tkeys, uint64_t n_tiles,
                                                 uint32_t* __restrict__ khk, uint64_t* __restrict__ kstart) {
    __shared__ uint32_t wsx[NWARP];
    const int w = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint64_t base = tile * FIN_TILE + (uint64_t)w * 32 * FIN_ITEMS + lane;
        uint32_t smask = 0, ns = 0;
        uint64_t v[FIN_ITEMS];
#pragma unroll
        for (int i = 0; i < FIN_ITEMS; ++i) {
            bool st, kept, over;
            fin_flags(a, n, 0xFFFFFFFFu, base + (uint64_t)i * 32, v[i], st, kept, over);
            smask |= (st ? 1u : 0u) << i;
            ns += __popc(__ballot_sync(FULL_MASK, st));
        }
        if (lane == 0) wsx[w] = ns;
        __syncthreads();
        uint64_t kidx = tkeys[tile];
        for (int i = 0; i < w; ++i) kidx += wsx[i];
        __syncthreads();
#pragma unroll
        for (int i = 0; i < FIN_ITEMS; ++i) {
            const bool st = (smask >> i) & 1u;
            const uint32_t bs = __ballot_sync(FULL_MASK, st);
            if (st) {
                const uint64_t my_s = kidx + __popc(bs & lt);
                khk[my_s] = hk_of(v[i]);
                kstart[my_s] = base + (uint64_t)i * 32;
            }
            kidx += __popc(bs);
        }
    }
}

// counts[i] = min(cap, length of run i); kstart has n_runs + 1 entries.
__global__ void k_run_counts(const uint64_t* __restrict__ kstart, uint64_t n_runs, uint32_t cap,
                             uint32_t* __restrict__ counts) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_runs;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t len = kstart[i + 1] - kstart[i];
        counts[i] = (uint32_t)(len < cap ? len : cap);
    }
}

// One list of earlier shards' feature counts (keys ascending).
struct PriorList {
    const uint32_t* keys;
    const uint32_t* counts;
    uint64_t n;
};

// Per run (thread per run): prior = the run's feature counts in the prior
// lists (binary search in each), limit = max(0, cap - prior); pairs of the
// run beyond the limit become sentinels.  Counts features whose locations
// together with the prior ones exceed cap.
__global__ void k_prior_limits(uint64_t* __restrict__ a, const uint32_t* __restrict__ khk,
                               const uint64_t* __restrict__ kstart, uint64_t n_runs, uint32_t cap,
                               const PriorList* __restrict__ lists, uint32_t n_lists,
                               unsigned long long* overflow) {
    unsigned long long n_over = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n_runs;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t key = khk[i];
        uint64_t prior = 0;
        for (uint32_t l = 0; l < n_lists; ++l) {
            const PriorList L = lists[l];
            uint64_t lo = 0, hi = L.n;  // first index with keys >= key
            while (lo < hi) {
                const uint64_t mid = (lo + hi) >> 1;
                if (L.keys[mid] < key) lo = mid + 1; else hi = mid;
            }
            if (lo < L.n && L.keys[lo] == key) prior += L.counts[lo];
        }
        if (prior == 0) continue;  // the plain cap applies
        const uint64_t len = kstart[i + 1] - kstart[i];
        const uint64_t limit = prior >= cap ? 0 : cap - prior;
        if (prior + len > cap) ++n_over;
        for (uint64_t e = kstart[i] + limit; e < kstart[i] + len; ++e) a[e] = SENTINEL_PAIR;
    }
    for (int o = 16; o >= 1; o >>= 1) n_over += __shfl_xor_sync(FULL_MASK, n_over, o);
    if (lane_id() == 0 && n_over) atomicAdd(overflow, n_over);
}

// Run starts of sorted pairs a[0..n): *n_runs, and (when keys != null and
// the runs fit max) keys[i], kstart[i] (n_runs + 1 entries, kstart[n_runs]
// = n) allocated by the caller.
cudaError_t sorted_runs(const Mem& mem, const uint64_t* a, uint64_t n, uint64_t max, uint32_t* keys,
                        uint64_t* kstart, uint64_t* n_runs, cudaStream_t s) {
    cudaError_t e;
    *n_runs = 0;
    if (n == 0) return cudaSuccess;
    const uint64_t tiles = (n + FIN_TILE - 1) / FIN_TILE;
    Tmp<uint64_t> tkept(mem, tiles + 1, s), tkeys(mem, tiles + 1, s);
    if (!tkept.ok() || !tkeys.ok()) return cudaErrorMemoryAllocation;
    MC_LAUNCH("fin_count", s, k_fin_count<<<grid_for(tiles), BT, 0, s>>>(a, n, 0xFFFFFFFFu, tkept.ptr, tkeys.ptr, tiles));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = scan_exclusive_sum(mem, tkeys.ptr, tkeys.ptr, tiles, s)) != cudaSuccess) return e;
    uint64_t total = 0;
    if ((e = cudaMemcpyAsync(&total, tkeys.ptr + tiles, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *n_runs = total;
    if (!keys || total > max) return cudaSuccess;
    MC_LAUNCH("run_emit", s, k_run_emit<<<grid_for(tiles), BT, 0, s>>>(a, n, tkeys.ptr, tiles, keys, kstart));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaMemcpyAsync(kstart + total, &n, 8, cudaMemcpyHostToDevice, s);
}
}  // namespace

cudaError_t feature_counts(const Mem& mem, const uint64_t* a, uint64_t n, uint32_t cap, uint64_t max, uint32_t* keys,
                           uint32_t* counts, uint64_t* n_keys, cudaStream_t s) {
    uint64_t runs = 0;
    cudaError_t e = sorted_runs(mem, a, n, 0, nullptr, nullptr, &runs, s);
    *n_keys = runs;
    if (e != cudaSuccess || runs == 0 || runs > max || !keys || !counts) return e;
    Tmp<uint64_t> kstart(mem, runs + 1, s);
    if (!kstart.ok()) return cudaErrorMemoryAllocation;
    uint64_t again = 0;
    if ((e = sorted_runs(mem, a, n, runs, keys, kstart.ptr, &again, s)) != cudaSuccess) return e;
    MC_LAUNCH("run_counts", s,
              k_run_counts<<<grid_for((runs + BT - 1) / BT), BT, 0, s>>>(kstart.ptr, runs, cap, counts));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

cudaError_t apply_prior(const Mem& mem, uint64_t* a, uint64_t n, uint32_t cap, uint32_t n_lists,
                        const uint32_t* const* keys, const uint32_t* const* counts, const uint64_t* list_n,
                        uint64_t* overflow, cudaStream_t s) {
    cudaError_t e;
    *overflow = 0;
    if (n == 0 || n_lists == 0) return cudaSuccess;
    uint64_t runs = 0;
    if ((e = sorted_runs(mem, a, n, 0, nullptr, nullptr, &runs, s)) != cudaSuccess) return e;
    Tmp<uint32_t> khk(mem, runs, s);
    Tmp<uint64_t> kstart(mem, runs + 1, s);
    Tmp<PriorList> dl(mem, n_lists, s);
    Tmp<unsigned long long> ctr(mem, 1, s);
    if (!khk.ok() || !kstart.ok() || !dl.ok() || !ctr.ok()) return cudaErrorMemoryAllocation;
    std::vector<PriorList> hl(n_lists);
    for (uint32_t l = 0; l < n_lists; ++l) hl[l] = PriorList{keys[l], counts[l], list_n[l]};
    uint64_t again = 0;
    if ((e = sorted_runs(mem, a, n, runs, khk.ptr, kstart.ptr, &again, s)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(dl.ptr, hl.data(), n_lists * sizeof(PriorList), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(ctr.ptr, 0, 8, s)) != cudaSuccess) return e;
    MC_LAUNCH("prior_limits", s,
              k_prior_limits<<<grid_for((runs + BT - 1) / BT), BT, 0, s>>>(a, khk.ptr, kstart.ptr, runs, cap, dl.ptr,
                                                                           n_lists, ctr.ptr));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned long long h = 0;
    if ((e = cudaMemcpyAsync(&h, ctr.ptr, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    *overflow = h;
    return cudaSuccess;
}

// -------------------------------------------------------------- taxonomy
namespace {
__global__ void k_tax_depth(const uint32_t* __restrict__ parent, uint32_t n, uint32_t* __restrict__ depth,
                            uint32_t* max_depth, uint32_t* cycle) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        uint32_t d = 0, y = x;
        while (parent[y] != y) {
            y = parent[y];
            if (++d > n) {
                atomicMax(cycle, 1u);
                d = 0;
                break;
            }
        }
        depth[x] = d;
        atomicMax(max_depth, d);
    }
}

__global__ void k_tax_lineage(const uint32_t* __restrict__ parent, uint32_t n, const uint32_t* __restrict__ depth,
                              uint32_t* __restrict__ lin, uint32_t stride) {
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        uint32_t y = x;
        for (int64_t d = depth[x]; d >= 0; --d) {
            lin[(uint64_t)x * stride + d] = y;
            y = parent[y];
        }
    }
}
}  // namespace

cudaError_t taxonomy_depths(const uint32_t* parent, uint32_t n_taxa, uint32_t* depth, uint32_t* max_depth,
                            uint32_t* cycle_flag, cudaStream_t s) {
    MC_LAUNCH("tax_depth", s, k_tax_depth<<<grid_for((n_taxa + BT - 1) / BT), BT, 0, s>>>(parent, n_taxa, depth, max_depth, cycle_flag));
    return cudaGetLastError();
}

cudaError_t taxonomy_lineage(const uint32_t* parent, uint32_t n_taxa, const uint32_t* depth, uint32_t* lin,
                             uint32_t stride, cudaStream_t s) {
    MC_LAUNCH("tax_lineage", s, k_tax_lineage<<<grid_for((n_taxa + BT - 1) / BT), BT, 0, s>>>(parent, n_taxa, depth, lin, stride));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ dump
namespace {
__global__ void k_dump_select(const uint64_t* __restrict__ table, uint64_t len, TableFmt fmt, uint64_t lo,
                              uint64_t hi, uint32_t* keys, uint64_t* offs, uint32_t* counts, uint64_t cap,
                              unsigned long long* n_sel) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < len; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t e = table[i];
        if (e == 0) continue;
        uint64_t key = hash_h2_inverse(fmt.key(e, i));
        if (key < lo || key >= hi) continue;
        unsigned long long idx = atomicAdd(n_sel, 1ull);
        if (idx < cap) {
            keys[idx] = (uint32_t)key;
            offs[idx] = fmt.offset(e);
            counts[idx] = fmt.count(e);
        }
    }
}

__global__ void k_dump_gather(const void* __restrict__ locs, uint32_t jbits, const uint64_t* __restrict__ src_off,
                              const uint32_t* __restrict__ counts, const uint64_t* __restrict__ dst_off, uint64_t n,
                              uint64_t* __restrict__ out) {
    for (uint64_t i = blockIdx.x; i < n; i += gridDim.x)
        for (uint32_t j = threadIdx.x; j < counts[i]; j += blockDim.x) {
            uint64_t v;
            if (jbits) {
                const uint32_t x = static_cast<const uint32_t*>(locs)[src_off[i] + j];
                v = ((uint64_t)(x >> jbits) << 32) | (x & ((1u << jbits) - 1u));
            } else {
                v = static_cast<const uint64_t*>(locs)[src_off[i] + j];
            }
            out[dst_off[i] + j] = v;
        }
}
}  // namespace

cudaError_t dump_select(const uint64_t* table, uint64_t table_len, TableFmt fmt, uint64_t lo, uint64_t hi,
                        uint32_t* keys, uint64_t* offs, uint32_t* counts, uint64_t cap, unsigned long long* n_sel,
                        cudaStream_t s) {
    if (table_len == 0) return cudaSuccess;
    MC_LAUNCH("dump_select", s,
              k_dump_select<<<grid_for((table_len + BT - 1) / BT), BT, 0, s>>>(table, table_len, fmt, lo, hi, keys,
                                                                               offs, counts, cap, n_sel));
    return cudaGetLastError();
}

cudaError_t dump_gather(const void* locs, uint32_t jbits, const uint64_t* src_off, const uint32_t* counts,
                        const uint64_t* dst_off, uint64_t n, uint64_t* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    MC_LAUNCH("dump_gather", s,
              k_dump_gather<<<grid_for(n, 32), 128, 0, s>>>(locs, jbits, src_off, counts, dst_off, n, out));
    return cudaGetLastError();
}

}  // namespace mc
