// Read classification kernels (Section 3.2 query phase, Section 4.2 query
// steps 1-8, Sections 4.3-4.6) for sm_103a.
//
// GB300 design.  The paper runs the query as a pipeline of kernels with
// global-memory hand-offs: sketch+lookup, compaction, a segmented sort
// (about half of its query time, Section 5.5) and a top-candidate kernel.
// Here one warp carries a whole query (a read or a read pair) through all
// steps without leaving the SM:
//   1. sketch every window of every mate (mc_sketch.cuh) and look each
//      feature up in the feature table (one 16-byte probe, Section 4.3);
//   2. gather the bucket locations into a per-warp hash histogram in shared
//      memory, location -> hit count (the window count statistic of
//      Section 3.2, replacing compaction + segmented sort + run-length
//      accumulation of Sections 4.4-4.6: order does not matter for counts);
//   3. score every distinct location (t, j0) as the sum of counts of
//      (t, j0 .. j0+sws-1) by histogram lookups (Section 4.6 sliding window);
//   4. keep per-lane top-m lists with one candidate per target, merge them
//      with warp shuffles (Section 4.6), and label the query by its top
//      target or the LCA of the close candidates via the lineage table.
// Queries whose histogram does not fit the shared-memory table (rare) are
// queued and processed by a second kernel whose warps use a larger table in
// global scratch memory.  Both paths run the same code, so the result does
// not depend on the path.
#include "mc_internal.h"
#include "mc_sketch.cuh"

namespace mc {

namespace {

constexpr int CLS_WARPS = 8;                 // warps per CTA
constexpr int WIN_A = 8;                     // windows per query on the shared-memory path
constexpr uint32_t KB_SLOTS = 1u << 16;      // large-path histogram slots per warp
constexpr uint32_t LIST_B = MC_MAX_QUERY_WINDOWS * MAX_S;
constexpr int B_WARPS_PER_SM = 2;

struct Cand {
    uint32_t score, t, j0, j1;
};

// Order of candidates: higher score first, then smaller target, then
// smaller first window (Section 3.2 top hits; ties are our reading).
__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.t != b.t) return a.t < b.t;
    return a.j0 < b.j0;
}

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int lane_mask) {
    Cand o;
    o.score = __shfl_xor_sync(FULL_MASK, c.score, lane_mask);
    o.t = __shfl_xor_sync(FULL_MASK, c.t, lane_mask);
    o.j0 = __shfl_xor_sync(FULL_MASK, c.j0, lane_mask);
    o.j1 = __shfl_xor_sync(FULL_MASK, c.j1, lane_mask);
    return o;
}

// Feature table lookup: ordered linear probing from the home slot; entries
// are in ascending h2 order along the table, so the probe stops at an empty
// slot or a larger key.  Returns the bucket size (0 if absent).
__device__ __forceinline__ uint32_t table_find(const uint4* __restrict__ tab, uint32_t log_t, uint32_t max_probe,
                                               uint32_t hk, uint64_t& off) {
    uint64_t pos = log_t >= 32 ? hk : (hk >> (32 - log_t));
    for (uint32_t d = 0; d <= max_probe; ++d) {
        uint4 e = __ldg(tab + pos + d);
        if (e.y == 0 || e.x > hk) return 0;
        if (e.x == hk) {
            off = (uint64_t)e.z | ((uint64_t)e.w << 32);
            return e.y;
        }
    }
    return 0;
}

__device__ __forceinline__ uint32_t loc_slot(uint64_t loc, uint32_t mask) {
    uint64_t h = (loc ^ (loc >> 29)) * 0x9E3779B97F4A7C15ull;
    return (uint32_t)(h >> 32) & mask;
}

// Histogram insert (count + 1).  Returns false if the table is full.
__device__ __forceinline__ bool hist_insert(uint64_t* keys, uint32_t* cnts, uint32_t mask, uint64_t loc,
                                            bool& fresh) {
    uint32_t slot = loc_slot(loc, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint64_t k = *(volatile uint64_t*)(keys + slot);
        if (k == loc) {
            atomicAdd(cnts + slot, 1u);
            fresh = false;
            return true;
        }
        if (k == EMPTY_LOC) {
            unsigned long long prev =
                atomicCAS((unsigned long long*)(keys + slot), (unsigned long long)EMPTY_LOC, (unsigned long long)loc);
            if (prev == EMPTY_LOC || prev == loc) {
                atomicAdd(cnts + slot, 1u);
                fresh = prev == EMPTY_LOC;
                return true;
            }
        }
        slot = (slot + 1) & mask;
    }
    fresh = false;
    return false;
}

__device__ __forceinline__ uint32_t hist_count(const uint64_t* keys, const uint32_t* cnts, uint32_t mask,
                                               uint64_t loc) {
    uint32_t slot = loc_slot(loc, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        uint64_t k = keys[slot];
        if (k == loc) return cnts[slot];
        if (k == EMPTY_LOC) return 0;
        slot = (slot + 1) & mask;
    }
    return 0;
}

// Per-lane top-m list with at most one candidate per target.
struct TopList {
    Cand c[MAX_M];
    int n;
    __device__ __forceinline__ void init() {
        n = 0;
#pragma unroll
        for (int i = 0; i < MAX_M; ++i) c[i] = Cand{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0};
    }
    __device__ __forceinline__ void remove_at(int idx) {
#pragma unroll
        for (int i = 0; i < MAX_M - 1; ++i)
            if (i >= idx) c[i] = c[i + 1];
        c[MAX_M - 1] = Cand{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0};
        --n;
    }
    __device__ __forceinline__ void insert(const Cand& x, int m) {
        if (n == m) {
            Cand last = c[0];
#pragma unroll
            for (int i = 0; i < MAX_M; ++i)
                if (i == m - 1) last = c[i];
            if (!better(x, last)) return;
        }
        int same = -1;
#pragma unroll
        for (int i = 0; i < MAX_M; ++i)
            if (i < n && c[i].t == x.t) same = i;
        if (same >= 0) {
            Cand old = c[0];
#pragma unroll
            for (int i = 0; i < MAX_M; ++i)
                if (i == same) old = c[i];
            if (!better(x, old)) return;
            remove_at(same);
        }
        if (n == m) {  // drop the last
#pragma unroll
            for (int i = 0; i < MAX_M; ++i)
                if (i == m - 1) c[i] = Cand{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0};
            --n;
        }
#pragma unroll
        for (int i = 0; i < MAX_M; ++i)
            if (i == n) c[i] = x;
        ++n;
#pragma unroll
        for (int i = MAX_M - 1; i >= 1; --i) {
            if (i < n && better(c[i], c[i - 1])) {
                Cand t = c[i];
                c[i] = c[i - 1];
                c[i - 1] = t;
            }
        }
    }
    __device__ __forceinline__ void remove_target(uint32_t t) {
        int idx = -1;
#pragma unroll
        for (int i = 0; i < MAX_M; ++i)
            if (i < n && c[i].t == t) idx = i;
        if (idx >= 0) remove_at(idx);
    }
};

__device__ __forceinline__ uint32_t lca2(const ClassifyDb& db, uint32_t a, uint32_t b) {
    if (a >= db.n_taxa || b >= db.n_taxa) return NO_TAXON;
    uint32_t da = db.depth[a], dbb = db.depth[b];
    int64_t d = da < dbb ? da : dbb;
    const uint32_t* la = db.lineage + (uint64_t)a * db.lin_stride;
    const uint32_t* lb = db.lineage + (uint64_t)b * db.lin_stride;
    for (; d >= 0; --d)
        if (la[d] == lb[d]) return la[d];
    return NO_TAXON;
}

enum { Q_DONE = 0, Q_ESCALATE = 1, Q_TOO_LARGE = 2 };

struct Scratch {
    uint64_t* keys;
    uint32_t* cnts;
    uint32_t kcap;  // power of two
    uint64_t* l_off;
    uint32_t* l_cnt;
    uint32_t* l_pre;  // list_cap + 1
    uint32_t list_cap;
    uint32_t win_cap;
};

// Lane i (< m) writes candidate slot i; `mine` is the lane's candidate.
__device__ __forceinline__ void write_result(const ClassifyQuery& Q, uint32_t q, uint32_t label, uint32_t hits,
                                             uint32_t top, const Cand& mine) {
    const uint32_t lane = lane_id();
    if (lane == 0) {
        Q.label[q] = label;
        Q.hits[q] = hits;
        if (Q.top_target) Q.top_target[q] = top;
    }
    if (Q.cands && lane < Q.m) {
        uint32_t* o = Q.cands + ((uint64_t)q * Q.m + lane) * 4;
        o[0] = mine.score;
        o[1] = mine.t;
        o[2] = mine.j0;
        o[3] = mine.j1;
    }
}

__device__ __forceinline__ void write_unclassified(const ClassifyQuery& Q, uint32_t q) {
    write_result(Q, q, NO_TAXON, 0, 0xFFFFFFFFu, Cand{0, 0xFFFFFFFFu, 0, 0});
}

template <int R>
__device__ __forceinline__ int process_query(const ClassifyDb& db, const ClassifyQuery& Q, uint32_t q, const Scratch& S,
                             unsigned long long (&ctr)[5]) {
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    const SketchParams& p = db.sp;
    const uint32_t m0 = Q.qoffs[q], m1 = Q.qoffs[q + 1];

    uint64_t span_sum = 0, n_win = 0;
    for (uint32_t i = m0; i < m1; ++i) {
        uint64_t L = Q.offs[i + 1] - Q.offs[i];
        span_sum += L;
        n_win += num_windows(L, p.k, p.stride);
    }
    if (n_win > MC_MAX_QUERY_WINDOWS) return Q_TOO_LARGE;
    if (n_win > S.win_cap) return Q_ESCALATE;

    // 1. sketch + lookup: list of (bucket offset, size) of found features
    uint32_t n_list = 0;
    uint64_t n_feat = 0, n_sect = 0;
    for (uint32_t i = m0; i < m1; ++i) {
        uint64_t L = Q.offs[i + 1] - Q.offs[i];
        uint64_t nw = num_windows(L, p.k, p.stride);
        const uint8_t* s = Q.seq + Q.offs[i];
        for (uint64_t j = 0; j < nw; ++j) {
            uint32_t f;
            uint32_t cnt = warp_sketch<R>(s, L, j * p.stride, p, f);
            n_feat += cnt;
            uint64_t off = 0;
            uint32_t c = 0;
            if (lane < cnt) c = table_find(db.table, db.log_t, db.max_probe, hash_h2(f), off);
            uint32_t found = __ballot_sync(FULL_MASK, c > 0);
            if (c > 0) {
                uint32_t idx = n_list + __popc(found & lt);
                S.l_off[idx] = off;
                S.l_cnt[idx] = c;
                // 32-byte sectors the bucket occupies (for the roofline counters)
                n_sect += ((off * 8 + (uint64_t)c * 8 - 1) >> 5) - ((off * 8) >> 5) + 1;
            }
            n_list += __popc(found);
        }
    }
    __syncwarp();

    // 2. exclusive prefix of bucket sizes; H = locations to gather
    uint32_t H = 0;
    for (uint32_t base = 0; base < n_list; base += 32) {
        uint32_t idx = base + lane;
        uint32_t c = idx < n_list ? S.l_cnt[idx] : 0;
        uint32_t inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t o = __shfl_up_sync(FULL_MASK, inc, d);
            if ((int)lane >= d) inc += o;
        }
        if (idx < n_list) S.l_pre[idx] = H + inc - c;
        H += __shfl_sync(FULL_MASK, inc, 31);
    }
    if (lane == 0) S.l_pre[n_list] = H;
    uint32_t kq = 32;
    while (kq < 2 * H && kq < S.kcap) kq <<= 1;
    const uint32_t mask = kq - 1;
    for (uint32_t s = lane; s < kq; s += 32) {
        S.keys[s] = EMPTY_LOC;
        S.cnts[s] = 0;
    }
    __syncwarp();

    // gather into the histogram
    const uint32_t limit = kq - kq / 8;
    uint32_t distinct = 0;
    uint32_t b = 0;
    for (uint32_t base = 0; base < H; base += 32) {
        uint32_t x = base + lane;
        bool fresh = false, ok = true;
        if (x < H) {
            while (S.l_pre[b + 1] <= x) ++b;
            uint64_t loc = db.locs[S.l_off[b] + (x - S.l_pre[b])];
            ok = hist_insert(S.keys, S.cnts, mask, loc, fresh);
        }
        distinct += __popc(__ballot_sync(FULL_MASK, fresh));
        if (__any_sync(FULL_MASK, !ok) || distinct > limit) return Q_ESCALATE;
    }
    __syncwarp();
    ctr[0] += n_feat;
    ctr[1] += H;
    ctr[2] += distinct;
    ctr[3] += n_list;
    ctr[4] += n_sect;  // per lane; summed over the warp at flush

    // 3. sliding-window scores (Section 4.6)
    uint64_t span = (m1 - m0 <= 1) ? span_sum : (span_sum > Q.max_insert ? span_sum : (uint64_t)Q.max_insert);
    uint32_t sws = span >= p.k ? (uint32_t)((span - p.k + p.stride - 1) / p.stride + 1) : 0;
    TopList tl;
    tl.init();
    const int m = (int)Q.m;
    for (uint32_t s = lane; s < kq; s += 32) {
        uint64_t loc = S.keys[s];
        if (loc == EMPTY_LOC) continue;
        Cand c;
        c.score = S.cnts[s];
        c.t = (uint32_t)(loc >> 32);
        c.j0 = (uint32_t)loc;
        c.j1 = c.j0;
        for (uint32_t d = 1; d < sws; ++d) {
            uint32_t n = hist_count(S.keys, S.cnts, mask, loc + d);
            if (n) {
                c.score += n;
                c.j1 = c.j0 + d;
            }
        }
        tl.insert(c, m);
    }

    // 4. warp merge of the lane lists: m rounds of arg-max, removing the
    // winner's target from every list.  Round r's winner is kept by lane r;
    // the close candidates' taxa are folded into the label as they come.
    Cand mine = Cand{0, 0xFFFFFFFFu, 0, 0};
    uint32_t label = NO_TAXON, hits = 0, top = 0xFFFFFFFFu;
    uint64_t bar = 0;
#pragma unroll
    for (int r = 0; r < MAX_M; ++r) {
        if (r >= m) break;
        Cand h = tl.n > 0 ? tl.c[0] : Cand{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0};
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            Cand x = shfl_cand(h, o);
            if (better(x, h)) h = x;
        }
        if (h.score == 0) break;
        if ((int)lane == r) mine = h;
        tl.remove_target(h.t);
        // 5. label (Section 3.2; hit threshold of Section 5.6)
        if (r == 0) {
            hits = h.score;
            top = h.t;
            bar = (uint64_t)(100 - Q.band) * hits;
            if (hits >= Q.hits_min) label = top < db.n_targets ? db.taxon_of_target[top] : NO_TAXON;
        } else if (hits >= Q.hits_min && 100ull * h.score >= bar) {
            uint32_t tx = h.t < db.n_targets ? db.taxon_of_target[h.t] : NO_TAXON;
            label = lca2(db, label, tx);
        }
    }
    write_result(Q, q, label, hits, top, mine);
    return Q_DONE;
}

// counters: [0] features looked up, [1] locations gathered, [2] distinct
// locations, [3] queries on the large path, [4] features found, [5] 32-byte
// sectors of the gathered buckets.
__device__ __forceinline__ void flush_counters(const ClassifyQuery& Q, unsigned long long (&ctr)[5]) {
    unsigned long long sect = ctr[4];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) sect += __shfl_xor_sync(FULL_MASK, sect, o);
    if (Q.counters && lane_id() == 0) {
        atomicAdd(Q.counters + 0, ctr[0]);
        atomicAdd(Q.counters + 1, ctr[1]);
        atomicAdd(Q.counters + 2, ctr[2]);
        atomicAdd(Q.counters + 4, ctr[3]);
        atomicAdd(Q.counters + 5, sect);
    }
}

// Shared-memory path: one warp per query, KA histogram slots per warp.
template <int R, int KA>
__global__ void __launch_bounds__(CLS_WARPS * 32, 1) k_classify_smem(ClassifyDb db, ClassifyQuery Q, uint32_t list_cap,
                                                                  uint32_t* __restrict__ ovf_list,
                                                                  uint32_t* __restrict__ ovf_n) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5;
    const size_t per_warp = (size_t)KA * 12 + (size_t)list_cap * 12 + (list_cap + 1) * 4 + 16;
    unsigned char* base = smem + w * ((per_warp + 15) & ~(size_t)15);
    Scratch S;
    S.keys = reinterpret_cast<uint64_t*>(base);
    S.l_off = reinterpret_cast<uint64_t*>(base + (size_t)KA * 8);
    S.cnts = reinterpret_cast<uint32_t*>(base + (size_t)KA * 8 + (size_t)list_cap * 8);
    S.l_cnt = S.cnts + KA;
    S.l_pre = S.l_cnt + list_cap;
    S.kcap = KA;
    S.list_cap = list_cap;
    S.win_cap = WIN_A;
    unsigned long long ctr[5] = {0, 0, 0, 0, 0};
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t q = gw; q < Q.n_q; q += nw) {
        int r = process_query<R>(db, Q, q, S, ctr);
        if (r == Q_ESCALATE) {
            if (lane_id() == 0) ovf_list[atomicAdd(ovf_n, 1u)] = q;
        } else if (r == Q_TOO_LARGE) {
            write_unclassified(Q, q);
            if (lane_id() == 0) atomicMax(Q.status, DEV_ERR_CAPACITY);
        }
        __syncwarp();
    }
    flush_counters(Q, ctr);
}

// Large path: queries queued by the shared-memory path, one warp each, with
// a KB_SLOTS histogram in global scratch memory.
template <int R>
__global__ void __launch_bounds__(CLS_WARPS * 32, 1) k_classify_large(ClassifyDb db, ClassifyQuery Q,
                                                                   const uint32_t* __restrict__ ovf_list,
                                                                   const uint32_t* __restrict__ ovf_n,
                                                                   uint32_t* __restrict__ work, uint64_t* gkeys,
                                                                   uint32_t* gcnts, uint64_t* gloff, uint32_t* glcnt,
                                                                   uint32_t* glpre) {
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    Scratch S;
    S.keys = gkeys + (uint64_t)gw * KB_SLOTS;
    S.cnts = gcnts + (uint64_t)gw * KB_SLOTS;
    S.kcap = KB_SLOTS;
    S.l_off = gloff + (uint64_t)gw * LIST_B;
    S.l_cnt = glcnt + (uint64_t)gw * LIST_B;
    S.l_pre = glpre + (uint64_t)gw * (LIST_B + 1);
    S.list_cap = LIST_B;
    S.win_cap = MC_MAX_QUERY_WINDOWS;
    unsigned long long ctr[5] = {0, 0, 0, 0, 0};
    const uint32_t n = *ovf_n;
    unsigned long long n_large = 0;
    for (;;) {
        uint32_t i = 0;
        if (lane_id() == 0) i = atomicAdd(work, 1u);
        i = __shfl_sync(FULL_MASK, i, 0);
        if (i >= n) break;
        uint32_t q = ovf_list[i];
        ++n_large;
        int r = process_query<R>(db, Q, q, S, ctr);
        if (r != Q_DONE) {
            write_unclassified(Q, q);
            if (lane_id() == 0) atomicMax(Q.status, DEV_ERR_CAPACITY);
        }
        __syncwarp();
    }
    flush_counters(Q, ctr);
    if (Q.counters && lane_id() == 0 && n_large) atomicAdd(Q.counters + 3, n_large);
}

constexpr int KA_DEFAULT = 512;

template <int R>
cudaError_t launch_all(const Mem& mem, const ClassifyDb& db, const ClassifyQuery& Q, cudaStream_t s) {
    cudaError_t e;
    const uint32_t list_cap = WIN_A * db.sp.s;
    const size_t per_warp = (size_t)KA_DEFAULT * 12 + (size_t)list_cap * 12 + (list_cap + 1) * 4 + 16;
    const size_t smem = CLS_WARPS * ((per_warp + 15) & ~(size_t)15);
    auto ka = k_classify_smem<R, KA_DEFAULT>;
    if ((e = cudaFuncSetAttribute(ka, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int dev = 0, sms = NUM_SMS_HINT, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ka, CLS_WARPS * 32, smem)) != cudaSuccess) return e;
    if (occ < 1) occ = 1;

    // scratch: overflow queue + counters
    Tmp<uint32_t> ovf(mem, (size_t)Q.n_q + 4, s);
    if (!ovf.ok()) return cudaErrorMemoryAllocation;
    uint32_t* ovf_n = ovf.ptr + Q.n_q;
    uint32_t* work = ovf_n + 1;
    if ((e = cudaMemsetAsync(ovf_n, 0, 2 * sizeof(uint32_t), s)) != cudaSuccess) return e;

    uint64_t blocks = ((uint64_t)Q.n_q + CLS_WARPS - 1) / CLS_WARPS;
    uint64_t cap_blocks = (uint64_t)sms * occ * 8;
    uint32_t g = (uint32_t)(blocks < cap_blocks ? blocks : cap_blocks);
    if (g == 0) return cudaSuccess;
    MC_LAUNCH("classify_smem", s, ka<<<g, CLS_WARPS * 32, smem, s>>>(db, Q, list_cap, ovf.ptr, ovf_n));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    // large path (persistent warps, exits at once if nothing was queued)
    const uint32_t b_blocks = (uint32_t)sms * B_WARPS_PER_SM / CLS_WARPS > 0 ? (uint32_t)sms * B_WARPS_PER_SM / CLS_WARPS : 1;
    const uint64_t b_warps = (uint64_t)b_blocks * CLS_WARPS;
    Tmp<uint64_t> gkeys(mem, b_warps * KB_SLOTS, s), gloff(mem, b_warps * LIST_B, s);
    Tmp<uint32_t> gcnts(mem, b_warps * KB_SLOTS, s), glcnt(mem, b_warps * LIST_B, s),
        glpre(mem, b_warps * (LIST_B + 1), s);
    if (!gkeys.ok() || !gloff.ok() || !gcnts.ok() || !glcnt.ok() || !glpre.ok()) return cudaErrorMemoryAllocation;
    MC_LAUNCH("classify_large", s, k_classify_large<R><<<b_blocks, CLS_WARPS * 32, 0, s>>>(db, Q, ovf.ptr, ovf_n, work, gkeys.ptr, gcnts.ptr,
                                                           gloff.ptr, glcnt.ptr, glpre.ptr));
    return cudaGetLastError();
}

}  // namespace

cudaError_t classify_launch(const Mem& mem, const ClassifyDb& db, const ClassifyQuery& Q, cudaStream_t s) {
    if (Q.n_q == 0) return cudaSuccess;
    int r = sketch_r_for(db.sp.w);
    if (r == 4) return launch_all<4>(mem, db, Q, s);
    if (r == 8) return launch_all<8>(mem, db, Q, s);
    return launch_all<16>(mem, db, Q, s);
}

}  // namespace mc
