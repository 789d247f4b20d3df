// Read classification kernels (Section 4.2 query phase, Section 5.2 query
// steps 1-8, Sections 5.3-5.6) for sm_103a.
//
// GB300 design.  The paper runs the query as a pipeline of kernels with
// global-memory hand-offs: sketch+lookup, compaction, a segmented sort
// (about half of its query time, Section 6.4) and a top-candidate kernel.
// Here one warp carries a whole query (a read or a read pair) through all
// steps without leaving the SM:
//   1. sketch every window of every mate (mc_sketch.cuh) and look each
//      feature up in the feature table (one 16-byte probe, Section 5.3);
//   2. gather the bucket locations into a per-warp hash histogram in shared
//      memory, location -> hit count (the window count statistic of
//      Section 4.2, replacing compaction + segmented sort + run-length
//      accumulation of Sections 5.4-5.6: order does not matter for counts);
//   3. score every distinct location (t, j0) as the sum of counts of
//      (t, j0 .. j0+sws-1) by histogram lookups (Section 5.6 sliding window);
//   4. keep per-lane top-m lists with one candidate per target, merge them
//      with warp shuffles (Section 5.6), and label the query by its top
//      target or the LCA of the close candidates via the lineage table.
// Queries whose histogram does not fit the shared-memory table (rare) are
// queued and processed by a second kernel whose warps use a larger table in
// global scratch memory.  Both paths run the same code, so the result does
// not depend on the path.
#include <algorithm>
#include <type_traits>

#include "mc_internal.h"
#include "mc_sketch.cuh"

namespace mc {

namespace {

constexpr int CLS_WARPS = 4;                 // warps per CTA (score and large paths)
constexpr int LK_WARPS = 8;                  // warps per CTA (lookup path)
constexpr int WIN_A = 8;                     // windows per query on the shared-memory path
constexpr uint32_t KB_SLOTS = 1u << 16;      // large-path histogram slots per warp
constexpr uint32_t LIST_B = MC_MAX_QUERY_WINDOWS * MAX_S;
constexpr int B_WARPS_PER_SM = 2;
constexpr uint32_t KM_SLOTS = 2048;          // medium-path histogram slots per warp
constexpr int MED_WARPS = 2;                 // warps per CTA (medium path)
constexpr int SK_NW = 2;  // windows sketched together

struct Cand {
    uint32_t score, t, j0, j1;
};

// Order of candidates: higher score first, then smaller target, then
// smaller first window (Section 4.2 top hits; ties are our reading).
__device__ __forceinline__ bool better(const Cand& a, const Cand& b) {
    if (a.score != b.score) return a.score > b.score;
    if (a.t != b.t) return a.t < b.t;
    return a.j0 < b.j0;
}

__device__ __forceinline__ uint32_t loc_slot(uint64_t loc, uint32_t mask) {
    uint64_t h = (loc ^ (loc >> 29)) * 0x9E3779B97F4A7C15ull;
    return (uint32_t)(h >> 32) & mask;
}
__device__ __forceinline__ uint32_t loc_slot(uint32_t key, uint32_t mask) {
    uint32_t h = key * 0x9E3779B1u;
    return (h ^ (h >> 15)) & mask;
}

// Histogram keys.  A database stores its locations as 32-bit words target
// << jbits | window when every id fits, else as 64-bit words target << 32 |
// window (LocT).  The histogram keys a location by the stored word itself
// (KeyT == LocT), or, for 32-bit words, optionally by the 64-bit form (the
// wide-key launch shape).
template <class KeyT, class LocT = KeyT>
struct KeyCodec {
    static_assert(sizeof(KeyT) >= sizeof(LocT), "keys are at least as wide as locations");
    uint32_t jbits;
    __device__ __forceinline__ KeyT encode(LocT loc) const {
        if (sizeof(KeyT) == sizeof(LocT)) return (KeyT)loc;
        const uint32_t x = (uint32_t)loc;
        return (KeyT)(((uint64_t)(x >> jbits) << 32) | (x & ((1u << jbits) - 1u)));
    }
    __device__ __forceinline__ uint32_t target(KeyT k) const {
        return sizeof(KeyT) == 8 ? (uint32_t)((uint64_t)k >> 32) : (uint32_t)k >> jbits;
    }
    __device__ __forceinline__ uint32_t window(KeyT k) const {
        return sizeof(KeyT) == 8 ? (uint32_t)k : (uint32_t)k & ((1u << jbits) - 1u);
    }
    // windows after this key's window before the id field would overflow
    __device__ __forceinline__ uint32_t room(KeyT k) const {
        return sizeof(KeyT) == 8 ? 0xFFFFFFFFu - (uint32_t)k : ((1u << jbits) - 1u) - window(k);
    }
    static constexpr KeyT empty() { return (KeyT)~(KeyT)0; }
};

__device__ __forceinline__ uint64_t key_cas(uint64_t* p, uint64_t cmp, uint64_t val) {
    return atomicCAS((unsigned long long*)p, (unsigned long long)cmp, (unsigned long long)val);
}
__device__ __forceinline__ uint32_t key_cas(uint32_t* p, uint32_t cmp, uint32_t val) { return atomicCAS(p, cmp, val); }

// Histogram count increment: 32-bit counts use atomicAdd directly; 16-bit
// counts add 1 << 16*(slot&1) to the aligned 32-bit word holding them (a
// count never passes 65535 there, so the neighbour is not disturbed).
__device__ __forceinline__ void count_inc(uint32_t* cnts, uint32_t slot) { atomicAdd(cnts + slot, 1u); }
__device__ __forceinline__ void count_inc(uint16_t* cnts, uint32_t slot) {
    atomicAdd(reinterpret_cast<uint32_t*>(cnts) + (slot >> 1), 1u << ((slot & 1u) * 16));
}

// Histogram insert (count + 1).  `fresh_slot` receives the slot if the
// location was new, else stays -1.  Returns false if the table is full.
template <class CntT, class KeyT>
__device__ __forceinline__ bool hist_insert(KeyT* keys, CntT* cnts, uint32_t mask, KeyT key, int& fresh_slot) {
    constexpr KeyT EMPTY = KeyCodec<KeyT>::empty();
    uint32_t slot = loc_slot(key, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        KeyT k = *(volatile KeyT*)(keys + slot);
        if (k == key) {
            count_inc(cnts, slot);
            return true;
        }
        if (k == EMPTY) {
            const KeyT prev = key_cas(keys + slot, EMPTY, key);
            if (prev == EMPTY || prev == key) {
                count_inc(cnts, slot);
                if (prev == EMPTY) fresh_slot = (int)slot;
                return true;
            }
        }
        slot = (slot + 1) & mask;
    }
    return false;
}

template <class CntT, class KeyT>
__device__ __forceinline__ uint32_t hist_count(const KeyT* keys, const CntT* cnts, uint32_t mask, KeyT key) {
    constexpr KeyT EMPTY = KeyCodec<KeyT>::empty();
    uint32_t slot = loc_slot(key, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const KeyT k = keys[slot];
        if (k == key) return cnts[slot];
        if (k == EMPTY) return 0;
        slot = (slot + 1) & mask;
    }
    return 0;
}

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

constexpr uint32_t MAX_MATES = MC_MAX_QUERY_MATES;  // mates per query (lane i holds mate i)
constexpr int LB_DEFAULT = 4;       // feature-table probes in flight per lane
constexpr int GB_DEFAULT = 8;       // bucket loads in flight per lane

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Per-warp working memory (shared memory on the main path, global scratch
// on the large path).  CntT is the histogram count type: 16 bits on the
// shared-memory path (whose queries gather at most 65,535 locations), 32
// bits on the large path.  Unused regions have size 0.
template <class CntT, class KeyT = uint64_t>
struct Scratch {
    KeyT* keys;        // histogram keys (location), kcap
    CntT* cnts;        // histogram counts, kcap
    CntT* score;       // sliding-window scores of the dense entries, kcap
    uint16_t* dense;   // slots of the distinct locations, kcap
    uint32_t kcap;     // power of two, <= 65536
    uint64_t* list;    // found buckets, offset << 16 | size, list_cap
    uint32_t* l_pre;   // exclusive prefix of bucket sizes, list_cap + 1
    uint32_t list_cap;
    uint32_t* feat;    // features of all windows, feat_cap
    uint32_t* cand;    // sketch selection scratch, SK_NW * 32
    uint8_t* buf;      // the query's bases, buf_cap
    uint32_t buf_cap;
    uint32_t win_cap;  // windows per query
    uint32_t max_locs; // locations per query
};

template <class CntT, class KeyT = uint64_t>
__host__ __device__ constexpr size_t scratch_bytes(uint32_t kcap, uint32_t list_cap, uint32_t feat_cap,
                                                   uint32_t buf_cap) {
    return align16((size_t)kcap * sizeof(KeyT)) + 2 * align16((size_t)kcap * sizeof(CntT)) + align16((size_t)kcap * 2) +
           align16((size_t)list_cap * 8) + align16(((size_t)list_cap + 4) * 4) + align16((size_t)feat_cap * 4) +
           (feat_cap ? align16(4 * 32 * SK_NW) : 0) + (buf_cap ? align16(buf_cap + 16) : 0);
}

// Carves a Scratch out of `base` (16-byte aligned), in scratch_bytes order.
template <class CntT, class KeyT = uint64_t>
__device__ __forceinline__ Scratch<CntT, KeyT> carve(unsigned char* base, uint32_t kcap, uint32_t list_cap,
                                                     uint32_t feat_cap, uint32_t buf_cap, uint32_t win_cap) {
    Scratch<CntT, KeyT> S;
    unsigned char* p = base;
    S.keys = reinterpret_cast<KeyT*>(p);
    p += align16((size_t)kcap * sizeof(KeyT));
    S.cnts = reinterpret_cast<CntT*>(p);
    p += align16((size_t)kcap * sizeof(CntT));
    S.score = reinterpret_cast<CntT*>(p);
    p += align16((size_t)kcap * sizeof(CntT));
    S.dense = reinterpret_cast<uint16_t*>(p);
    p += align16((size_t)kcap * 2);
    S.list = reinterpret_cast<uint64_t*>(p);
    p += align16((size_t)list_cap * 8);
    S.l_pre = reinterpret_cast<uint32_t*>(p);
    p += align16(((size_t)list_cap + 4) * 4);
    S.feat = reinterpret_cast<uint32_t*>(p);
    p += align16((size_t)feat_cap * 4);
    S.cand = reinterpret_cast<uint32_t*>(p);
    p += feat_cap ? align16(4 * 32 * SK_NW) : 0;
    S.buf = p;
    S.kcap = kcap;
    S.list_cap = list_cap;
    S.buf_cap = buf_cap;
    S.win_cap = win_cap;
    S.max_locs = sizeof(CntT) == 2 ? 0xFFFFu : 0xFFFFFFFFu;
    return S;
}

struct Counters {
    unsigned long long features = 0, locations = 0, distinct = 0, found = 0, sectors = 0, queries = 0;
};

// Per-kernel counter block of mc_classify_debug: kernel k (0 hash score,
// 1-3 sort path 256/512/1024, 4 medium path, 5 large path, 6 sort path
// 2048) adds the queries it finished, their found buckets and their
// 32-byte sectors at counters[7 + 3k ...].
constexpr int KC_SCORE = 0, KC_MEDIUM = 4, KC_LARGE = 5;

// Batch holding query q of a multi-batch launch: the last batch whose
// first query is <= q (empty batches share their first query number with
// the next batch, so they are never chosen).
__device__ __forceinline__ uint32_t find_batch(const ClassifyQuery& Q, uint32_t q) {
    const uint32_t* pre = Q.bhdr + 2;
    uint32_t lo = 0, hi = Q.bhdr[0];
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= q) lo = mid; else hi = mid;
    }
    return lo;
}

// Number of queries of the launch (read on the device in the multi-batch
// form, so that a captured launch serves any batch set within capacity).
__device__ __forceinline__ uint32_t total_queries(const ClassifyQuery& Q) {
    return Q.batches ? Q.bhdr[1] : Q.n_q;
}

// Input of query q: its sequences and its mates' range.
struct QueryIn {
    const uint8_t* seq;
    const uint64_t* offs;
    uint32_t m0, m1;
};

__device__ __forceinline__ QueryIn query_in(const ClassifyQuery& Q, uint32_t q) {
    if (!Q.batches) return QueryIn{Q.seq, Q.offs, Q.qoffs[q], Q.qoffs[q + 1]};
    const uint32_t b = find_batch(Q, q);
    const BatchDesc& B = Q.batches[b];
    const uint32_t lq = q - Q.bhdr[2 + b];
    return QueryIn{B.seq, B.offs, B.qoffs[lq], B.qoffs[lq + 1]};
}

// Lane i (< m) writes candidate slot i; `mine` is the lane's candidate.
__device__ __forceinline__ void write_result(const ClassifyQuery& Q, uint32_t q, uint32_t label, uint32_t hits,
                                             uint32_t top, const Cand& mine) {
    const uint32_t lane = lane_id();
    if (lane == 0) {
        uint32_t* lab = Q.label;
        uint32_t* hit = Q.hits;
        uint32_t* tt = Q.top_target;
        uint32_t lq = q;
        if (Q.batches) {
            const uint32_t b = find_batch(Q, q);
            lab = Q.batches[b].label;
            hit = Q.batches[b].hits;
            tt = Q.batches[b].top_target;
            lq = q - Q.bhdr[2 + b];
        }
        lab[lq] = label;
        hit[lq] = hits;
        if (tt) tt[lq] = top;
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

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// 16-byte asynchronous copy global -> shared (completion: cp_async_wait_all).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// A query whose bases are (being) staged in working memory.  Per lane: the
// length, window count and staging offset of mate `lane`; the rest is
// warp-uniform.
struct Staged {
    int status;  // Q_DONE, Q_ESCALATE or Q_TOO_LARGE
    uint32_t nm, shift, span, n_win;
    uint32_t L, nw, boff;
};

// Query step 1a: reads the query's mates and stages its bases in buf (the
// mates of a query are consecutive sequences, so this is one contiguous
// range), placed at the same offset mod 16 as in memory.  ASYNC: every
// 16-byte aligned chunk that holds a base of the query is copied with
// cp.async (completion: cp_async_wait_all + __syncwarp; bytes of those
// chunks outside the query are copied too and never read).  Otherwise the
// aligned chunks inside the range are vector loads and the partial chunks
// at both ends are copied byte by byte.
template <bool ASYNC>
__device__ __forceinline__ Staged stage_query(const ClassifyDb& db, const ClassifyQuery& Q, uint32_t q, uint8_t* buf,
                                              uint32_t buf_cap, uint32_t win_cap) {
    const uint32_t lane = lane_id();
    const SketchParams& p = db.sp;
    Staged st{};
    const QueryIn in = query_in(Q, q);
    const uint32_t m0 = in.m0, m1 = in.m1;
    if (m1 < m0 || m1 - m0 > MAX_MATES) {
        st.status = Q_TOO_LARGE;
        return st;
    }
    const uint32_t nm = m1 - m0;
    // mates: lane i holds mate i's offset, length and window count
    const uint64_t o = lane <= nm ? in.offs[m0 + lane] : 0;
    const uint64_t o_next = __shfl_down_sync(FULL_MASK, o, 1);
    const uint64_t L = (lane < nm && o_next > o) ? o_next - o : 0;
    const uint64_t nw = lane < nm ? num_windows(L, p.k, p.stride) : 0;
    const uint64_t span_sum = warp_sum_u64(L);
    const uint64_t n_win = warp_sum_u64(nw);
    if (n_win > MC_MAX_QUERY_WINDOWS) {
        st.status = Q_TOO_LARGE;
        return st;
    }
    if (n_win > win_cap || span_sum > buf_cap) {
        st.status = Q_ESCALATE;
        return st;
    }
    uint64_t boff = L;  // exclusive prefix of mate lengths
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t x = __shfl_up_sync(FULL_MASK, boff, d);
        if ((int)lane >= d) boff += x;
    }
    boff -= L;
    const uint64_t start = __shfl_sync(FULL_MASK, o, 0);
    const uintptr_t first = (uintptr_t)(in.seq + start);
    const uint32_t shift = (uint32_t)(first & 15u);
    const uintptr_t a0 = first - shift;
    const uint64_t n_chunks = (shift + span_sum + 15) / 16;
    if (ASYNC) {
        for (uint64_t c = lane; c < n_chunks; c += 32)
            cp_async16(buf + 16 * c, reinterpret_cast<const void*>(a0 + 16 * c));
        cp_async_commit();
    } else {
        for (uint64_t c = lane; c < n_chunks; c += 32) {
            const uintptr_t cs = a0 + 16 * c;
            if (cs >= first && cs + 16 <= first + span_sum) {
                *reinterpret_cast<uint4*>(buf + 16 * c) = __ldg(reinterpret_cast<const uint4*>(cs));
            } else {
                const uintptr_t lo = cs > first ? cs : first;
                const uintptr_t hi = cs + 16 < first + span_sum ? cs + 16 : first + span_sum;
                for (uintptr_t b = lo; b < hi; ++b) buf[b - a0] = __ldg(reinterpret_cast<const uint8_t*>(b));
            }
        }
        __syncwarp();
    }
    st.status = Q_DONE;
    st.nm = nm;
    st.shift = shift;
    st.span = (uint32_t)span_sum;
    st.n_win = (uint32_t)n_win;
    st.L = (uint32_t)L;
    st.nw = (uint32_t)nw;
    st.boff = (uint32_t)boff;
    return st;
}

// Query steps 1b-4 of Section 5.2 on one warp, for a query staged in buf:
// sketch every window of every mate, look every feature up; the found
// buckets are written to `list` (working memory or global scratch), packed
// as offset << 16 | size.  Also returns the sliding-window size, the number
// of features and the 32-byte sectors of the found buckets (warp totals).
template <int R, int KC, int LB, class CntT>
__device__ __forceinline__ void sketch_probe(const ClassifyDb& db, const ClassifyQuery& Q, const Scratch<CntT>& S,
                                             const uint8_t* buf, const Staged& sq, uint64_t* __restrict__ list,
                                             uint32_t& n_list_out, uint32_t& sws_out, uint32_t& n_feat_out,
                                             uint32_t& n_sect_out, uint32_t& n_locs_out) {
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    const SketchParams& p = db.sp;
    const uint32_t nm = sq.nm, shift = sq.shift;
    const uint64_t L = sq.L, nw = sq.nw, boff = sq.boff, n_win = sq.n_win, span_sum = sq.span;

    // 1b. sketch every window of every mate (Section 4.2: reads are windowed
    // like the targets), SK_NW windows at a time; feat[] gets the features
    // in window order
    uint32_t F = 0;
    {
        uint32_t mi = 0;          // mate of the next window
        uint64_t jn = 0;          // its window index
        uint64_t nw_mi = __shfl_sync(FULL_MASK, nw, 0);
        for (uint64_t done = 0; done < n_win; done += SK_NW) {
            const uint8_t* sqp[SK_NW];
            uint64_t Ls[SK_NW], wss[SK_NW];
            bool act[SK_NW];
#pragma unroll
            for (int i = 0; i < SK_NW; ++i) {
                act[i] = done + i < n_win;
                while (act[i] && jn >= nw_mi) {  // skip to the mate of this window
                    ++mi;
                    jn = 0;
                    nw_mi = __shfl_sync(FULL_MASK, nw, mi & 31);
                }
                sqp[i] = buf + shift + __shfl_sync(FULL_MASK, boff, mi & 31);
                Ls[i] = act[i] ? __shfl_sync(FULL_MASK, L, mi & 31) : 0;
                wss[i] = jn * p.stride;
                if (act[i]) ++jn;
            }
            uint32_t f[SK_NW], cnt[SK_NW];
            warp_sketch_multi<R, SK_NW, KC, false>(sqp, Ls, wss, act, p, S.cand, f, cnt);
#pragma unroll
            for (int i = 0; i < SK_NW; ++i) {
                if (lane < cnt[i]) S.feat[F + lane] = f[i];
                F += cnt[i];
            }
        }
    }
    __syncwarp();

    // 1c. feature table probes, LB per lane in flight.  A probe reads the
    // aligned 16-byte pair of table words holding the home slot, then
    // follows the ordered probe sequence (stop at an empty slot or a key >=
    // h) one word at a time; the longest sequence is the table's largest
    // displacement.
    const TableFmt fmt = db.fmt;
    const uint32_t lsz = db.jbits ? 4u : 8u;  // bytes per stored location
    uint32_t n_list = 0;
    unsigned long long n_sect = 0, n_locs = 0;
    for (uint32_t base = 0; base < F; base += 32 * LB) {
        uint32_t hk[LB];
        uint64_t pos[LB];
        ulonglong2 pr[LB];
#pragma unroll
        for (int b = 0; b < LB; ++b) {
            const uint32_t idx = base + b * 32 + lane;
            hk[b] = idx < F ? hash_h2(S.feat[idx]) : 0u;
            pos[b] = fmt.home(hk[b]);
            pr[b] = idx < F ? __ldg(reinterpret_cast<const ulonglong2*>(db.table + (pos[b] & ~1ull)))
                            : make_ulonglong2(0, 0);
        }
#pragma unroll
        for (int b = 0; b < LB; ++b) {
            const uint32_t idx = base + b * 32 + lane;
            uint32_t c = 0;
            uint64_t off = 0;
            if (idx < F) {
                uint64_t slot = pos[b];
                uint64_t e = (slot & 1) ? pr[b].y : pr[b].x;
                for (uint32_t d = 0; e != 0; ) {
                    const uint32_t k = fmt.key(e, slot);
                    if (k >= hk[b]) {
                        if (k == hk[b]) {
                            c = fmt.count(e);
                            off = fmt.offset(e);
                        }
                        break;
                    }
                    if (++d > db.max_probe) break;
                    ++slot;
                    e = (slot == (pos[b] | 1ull)) ? pr[b].y : __ldg(db.table + slot);
                }
            }
            const uint32_t found = __ballot_sync(FULL_MASK, c > 0);
            if (c > 0) {
                list[n_list + __popc(found & lt)] = (off << 16) | c;
                n_sect += ((off * lsz + (uint64_t)c * lsz - 1) >> 5) - ((off * lsz) >> 5) + 1;
                n_locs += c;
            }
            n_list += __popc(found);
        }
    }
    __syncwarp();
    n_feat_out = F;
    n_sect_out = (uint32_t)warp_sum_u64(n_sect);
    n_locs_out = (uint32_t)warp_sum_u64(n_locs);  // <= 2048 features x 65535
    const uint64_t span = (nm <= 1) ? span_sum : (span_sum > Q.max_insert ? span_sum : (uint64_t)Q.max_insert);
    sws_out = span >= p.k ? (uint32_t)((span - p.k + p.stride - 1) / p.stride + 1) : 0;
    n_list_out = n_list;
}

// Query steps 1-4 on one warp (staging, sketch, lookup), synchronously.
// Returns Q_DONE, Q_ESCALATE (needs the large path) or Q_TOO_LARGE.
template <int R, int KC, int LB, class CntT>
__device__ __forceinline__ int query_lookup(const ClassifyDb& db, const ClassifyQuery& Q, uint32_t q,
                                            const Scratch<CntT>& S, uint64_t* __restrict__ list, uint32_t& n_list_out,
                                            uint32_t& sws_out, uint32_t& n_feat_out, uint32_t& n_sect_out) {
    const Staged st = stage_query<false>(db, Q, q, S.buf, S.buf_cap, S.win_cap);
    if (st.status != Q_DONE) return st.status;
    uint32_t n_locs = 0;
    sketch_probe<R, KC, LB>(db, Q, S, S.buf, st, list, n_list_out, sws_out, n_feat_out, n_sect_out, n_locs);
    return Q_DONE;
}

// Query steps 5-8 of Section 5.2 on one warp, from the bucket list in
// working memory: gather, window count statistic, sliding-window scores,
// top m, label.  Writes the outputs and returns Q_DONE, or Q_ESCALATE if the
// histogram does not fit the working memory.
template <int GB, class LocT, class CntT, class KeyT>
__device__ __forceinline__ int query_score(const ClassifyDb& db, const ClassifyQuery& Q, uint32_t q,
                                           const Scratch<CntT, KeyT>& S, uint32_t n_list, uint32_t sws,
                                           Counters& ctr) {
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
    const KeyCodec<KeyT, LocT> kc{db.jbits};
    constexpr KeyT EMPTY = KeyCodec<KeyT>::empty();
    constexpr LocT NO_LOC = (LocT)~(LocT)0;  // never a stored location
    const LocT* __restrict__ locs = static_cast<const LocT*>(db.locs);

    // 2. exclusive prefix of bucket sizes; H = locations to gather
    uint32_t H = 0;
    for (uint32_t base = 0; base < n_list; base += 32) {
        const uint32_t idx = base + lane;
        const uint32_t c = idx < n_list ? (uint32_t)(S.list[idx] & 0xFFFFu) : 0;
        uint32_t inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t x = __shfl_up_sync(FULL_MASK, inc, d);
            if ((int)lane >= d) inc += x;
        }
        if (idx < n_list) S.l_pre[idx] = H + inc - c;
        H += __shfl_sync(FULL_MASK, inc, 31);
    }
    if (lane == 0) S.l_pre[n_list] = H;
    if (H > S.max_locs) return Q_ESCALATE;
    uint32_t kq = 32;
    while (kq < 2 * H && kq < S.kcap) kq <<= 1;
    const uint32_t mask = kq - 1;
    for (uint32_t s = lane; s < kq; s += 32) {
        S.keys[s] = EMPTY;
        S.cnts[s] = 0;
    }
    __syncwarp();

    // 3. gather the buckets into the hit histogram (window count statistic,
    // Section 4.2): each lane loads GB consecutive locations of the flat
    // list (all in flight), then inserts them; the slots of new locations
    // are appended to a dense list
    // at most 3/4 of the slots in use: linear probing stays short (an absent
    // key costs about 8.5 probes at 3/4, 32 at 7/8)
    const uint32_t limit = kq - kq / 4;
    uint32_t D = 0;
    for (uint32_t base = 0; base < H; base += 32 * GB) {
        const uint32_t x0 = base + lane * GB;
        // bucket of x0: last b with l_pre[b] <= x0
        uint32_t lo = 0, hi = n_list;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (S.l_pre[mid] <= x0) lo = mid; else hi = mid;
        }
        uint32_t bkt = lo;
        LocT v[GB];
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            const uint32_t x = x0 + g;
            v[g] = NO_LOC;
            if (x < H) {
                while (S.l_pre[bkt + 1] <= x) ++bkt;
                v[g] = __ldg(locs + (S.list[bkt] >> 16) + (x - S.l_pre[bkt]));
            }
        }
        bool ok = true;
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            int slot = -1;
            if (v[g] != NO_LOC) ok &= hist_insert(S.keys, S.cnts, mask, kc.encode(v[g]), slot);
            const uint32_t fresh = __ballot_sync(FULL_MASK, slot >= 0);
            if (slot >= 0) S.dense[D + __popc(fresh & lt)] = (uint16_t)slot;
            D += __popc(fresh);
            // checked after every round, so the table never passes limit + 32
            // entries: inserts stay cheap and a query that will not fit is
            // handed on as soon as it is known
            if (D > limit) return Q_ESCALATE;
        }
        if (__any_sync(FULL_MASK, !ok)) return Q_ESCALATE;
    }
    __syncwarp();
    ctr.locations += H;
    ctr.distinct += D;

    // 4. sliding-window scores (Section 5.6): score(t, j0) = sum of the
    // counts of (t, j0 .. j0+sws-1), for the distinct locations
    for (uint32_t i = lane; i < D; i += 32) {
        const uint32_t slot = S.dense[i];
        const KeyT key = S.keys[slot];
        uint32_t sc = S.cnts[slot];
        const uint32_t room = kc.room(key);  // windows left before the id wraps
        for (uint32_t d = 1; d < sws && d <= room; ++d) sc += hist_count(S.keys, S.cnts, mask, (KeyT)(key + d));
        S.score[i] = (CntT)sc;
    }
    __syncwarp();

    // 5. top m with one candidate per target (Section 4.2 / 5.6): rounds of
    // warp arg-max; the winner's target is excluded from later rounds by
    // zeroing the scores of its entries.  The label is folded as the
    // candidates come (hit threshold of Section 6.5, LCA of the close
    // candidates of Section 4.2).  Later rounds only give lower scores, so
    // unless the full top-m list is requested the rounds stop once the
    // query is unclassified or the best remaining score is not close.
    const int m = (int)Q.m;
    Cand mine = Cand{0, 0xFFFFFFFFu, 0, 0};
    uint32_t label = NO_TAXON, hits = 0, top = 0xFFFFFFFFu;
    uint64_t bar = 0;
    uint32_t prev_t = 0xFFFFFFFFu;
    for (int r = 0; r < m; ++r) {
        Cand best = Cand{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0};
        for (uint32_t i = lane; i < D; i += 32) {
            uint32_t sc = S.score[i];
            if (sc == 0) continue;
            const KeyT key = S.keys[S.dense[i]];
            const uint32_t t = kc.target(key);
            if (t == prev_t) {
                S.score[i] = 0;
                continue;
            }
            const Cand c = Cand{sc, t, kc.window(key), 0};
            if (better(c, best)) best = c;
        }
        // warp arg-max in the candidate order: highest score, then smallest
        // target, then smallest first window
        {
            const uint32_t ms = __reduce_max_sync(FULL_MASK, best.score);
            const uint32_t mt = __reduce_min_sync(FULL_MASK, best.score == ms ? best.t : 0xFFFFFFFFu);
            const uint32_t mj =
                __reduce_min_sync(FULL_MASK, (best.score == ms && best.t == mt) ? best.j0 : 0xFFFFFFFFu);
            best = Cand{ms, mt, mj, 0};
        }
        if (best.score == 0) break;
        prev_t = best.t;
        if (Q.cands) {
            // last window of the range present in the histogram
            uint32_t j1 = best.j0;
            for (uint32_t i = lane; i < D; i += 32) {
                const KeyT key = S.keys[S.dense[i]];
                const uint32_t j = kc.window(key);
                if (kc.target(key) == best.t && j >= best.j0 && (uint64_t)j < (uint64_t)best.j0 + sws && j > j1)
                    j1 = j;
            }
            best.j1 = __reduce_max_sync(FULL_MASK, j1);
        }
        if ((int)lane == r) mine = best;
        if (r == 0) {
            hits = best.score;
            top = best.t;
            bar = (uint64_t)(100 - Q.band) * hits;
            if (hits >= Q.hits_min) label = top < db.n_targets ? db.taxon_of_target[top] : NO_TAXON;
            else if (!Q.cands) break;
        } else if (hits >= Q.hits_min && 100ull * best.score >= bar) {
            const uint32_t tx = best.t < db.n_targets ? db.taxon_of_target[best.t] : NO_TAXON;
            label = lca2(db, label, tx);
        } else if (!Q.cands) {
            break;
        }
        __syncwarp();
    }
    write_result(Q, q, label, hits, top, mine);
    return Q_DONE;
}

// Whole query on one warp with the bucket list in working memory.
template <int R, int KC, class LocT, class CntT>
__device__ __forceinline__ int process_query(const ClassifyDb& db, const ClassifyQuery& Q, uint32_t q,
                                             const Scratch<CntT>& S, Counters& ctr) {
    uint32_t n_list = 0, sws = 0, n_feat = 0, n_sect = 0;
    int r = query_lookup<R, KC, LB_DEFAULT>(db, Q, q, S, S.list, n_list, sws, n_feat, n_sect);
    if (r != Q_DONE) return r;
    r = query_score<GB_DEFAULT, LocT>(db, Q, q, S, n_list, sws, ctr);
    if (r == Q_DONE) {
        ctr.features += n_feat;
        ctr.found += n_list;
        ctr.sectors += n_sect;
        ++ctr.queries;
    }
    return r;
}

// counters: [0] features looked up, [1] locations gathered, [2] distinct
// locations, [3] queries on the large path, [4] features found, [5] 32-byte
// sectors of the gathered buckets, [6] queries finished on the medium path.
__device__ __forceinline__ void flush_counters(const ClassifyQuery& Q, const Counters& c, int kidx) {
    const unsigned long long sect = c.sectors;
    if (Q.counters && lane_id() == 0) {
        atomicAdd(Q.counters + 0, c.features);
        atomicAdd(Q.counters + 1, c.locations);
        atomicAdd(Q.counters + 2, c.distinct);
        atomicAdd(Q.counters + 4, c.found);
        atomicAdd(Q.counters + 5, sect);
        atomicAdd(Q.counters + 7 + 3 * kidx, c.queries);
        atomicAdd(Q.counters + 8 + 3 * kidx, c.found);
        atomicAdd(Q.counters + 9 + 3 * kidx, sect);
    }
}

constexpr uint32_t BUF_A = 1024;   // bases per query on the shared-memory path
constexpr uint32_t BUF_B = 16384;  // bases per query on the large path

constexpr uint32_t ESCALATED = 0xFFFFFFFFu;

// A Staged query kept in shared memory (per lane: L, nw, boff; then the
// warp-uniform fields).
constexpr size_t STAGED_BYTES = 3 * 32 * 4 + 8 * 4;

__device__ __forceinline__ void save_staged(unsigned char* rec, const Staged& st) {
    uint32_t* r = reinterpret_cast<uint32_t*>(rec);
    const uint32_t lane = lane_id();
    r[lane] = st.L;
    r[32 + lane] = st.nw;
    r[64 + lane] = st.boff;
    if (lane == 0) {
        r[96] = (uint32_t)st.status;
        r[97] = st.nm;
        r[98] = st.shift;
        r[99] = st.span;
        r[100] = st.n_win;
    }
}

__device__ __forceinline__ Staged load_staged(const unsigned char* rec) {
    const uint32_t* r = reinterpret_cast<const uint32_t*>(rec);
    const uint32_t lane = lane_id();
    Staged st;
    st.L = r[lane];
    st.nw = r[32 + lane];
    st.boff = r[64 + lane];
    st.status = (int)r[96];
    st.nm = r[97];
    st.shift = r[98];
    st.span = r[99];
    st.n_win = r[100];
    return st;
}

// Shared memory of one lookup warp: working memory, a second staging buffer
// and two staged-query records.
__host__ __device__ constexpr size_t lookup_warp_bytes(uint32_t list_cap) {
    return scratch_bytes<uint16_t>(0, 0, list_cap, BUF_A) + align16(BUF_A + 16) + 2 * STAGED_BYTES;
}

// Per-query metadata written by the lookup kernel: {found buckets, sliding
// window size | features << META_FEAT_SHIFT, locations to gather, 32-byte
// sectors of those locations}, or x = ESCALATED.  On this path a query has
// at most WIN_A * MAX_S = 256 features and a sliding window below 2^17.
constexpr uint32_t META_FEAT_SHIFT = 20;
__device__ __forceinline__ uint32_t meta_sws(const uint4& m) { return m.y & ((1u << META_FEAT_SHIFT) - 1u); }
__device__ __forceinline__ uint32_t meta_feat(const uint4& m) { return m.y >> META_FEAT_SHIFT; }

// Main path, part 1 (sketch + lookup): one warp per query of the chunk
// [q0, q0 + nq), shared memory for the query's bases and features only, so
// many warps fit on an SM.  Software-pipelined: the bases of the warp's
// next query are copied (cp.async) into the other staging buffer while the
// current query is sketched and looked up.  Writes each query's bucket list
// to glist[(q - q0) * list_cap ...] and {list size, sliding-window size} to
// meta; queries that need the large path are queued.
template <int R, int KC, int LB>
__global__ void __launch_bounds__(LK_WARPS * 32, 4) k_classify_lookup(ClassifyDb db, ClassifyQuery Q, uint32_t q0,
                                                                  uint32_t chunk, uint32_t list_cap,
                                                                  uint64_t* __restrict__ glist,
                                                                  uint4* __restrict__ meta,
                                                                  uint32_t* __restrict__ ovf_list,
                                                                  uint32_t* __restrict__ ovf_n) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5;
    unsigned char* mine = smem + w * lookup_warp_bytes(list_cap);
    const Scratch<uint16_t> S = carve<uint16_t>(mine, 0, 0, list_cap, BUF_A, WIN_A);
    uint8_t* const buf0 = S.buf;
    uint8_t* const buf1 = mine + scratch_bytes<uint16_t>(0, 0, list_cap, BUF_A);
    unsigned char* recs = buf1 + align16(BUF_A + 16);
    const uint32_t total = total_queries(Q);
    if (q0 >= total) return;
    const uint32_t nq = min(chunk, total - q0);
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarp = (gridDim.x * blockDim.x) >> 5;
    uint32_t cur = 0;
    if (gw < nq) save_staged(recs, stage_query<true>(db, Q, q0 + gw, buf0, BUF_A, WIN_A));
    for (uint32_t i = gw; i < nq; i += nwarp) {
        cp_async_wait_all();
        __syncwarp();
        const uint32_t nx = i + nwarp;
        if (nx < nq)
            save_staged(recs + (cur ^ 1) * STAGED_BYTES,
                        stage_query<true>(db, Q, q0 + nx, cur ? buf0 : buf1, BUF_A, WIN_A));
        const Staged st = load_staged(recs + cur * STAGED_BYTES);
        const uint32_t q = q0 + i;
        uint32_t n_list = 0, sws = 0, n_feat = 0, n_sect = 0, n_locs = 0;
        int r = st.status;
        if (r == Q_DONE)
            sketch_probe<R, KC, LB>(db, Q, S, cur ? buf1 : buf0, st, glist + (uint64_t)i * list_cap, n_list, sws, n_feat,
                                    n_sect, n_locs);
        if (r == Q_ESCALATE) {
            if (lane_id() == 0) {
                ovf_list[atomicAdd(ovf_n, 1u)] = q;
                meta[i] = make_uint4(ESCALATED, 0, 0, 0);
            }
        } else if (r == Q_TOO_LARGE) {
            write_unclassified(Q, q);
            if (lane_id() == 0) {
                atomicMax(Q.status, DEV_ERR_CAPACITY);
                meta[i] = make_uint4(ESCALATED, 0, 0, 0);
            }
        } else if (lane_id() == 0) {
            meta[i] = make_uint4(n_list, sws | (n_feat << META_FEAT_SHIFT), n_locs, n_sect);
        }
        __syncwarp();
        cur ^= 1;
    }
    cp_async_wait_all();
}

// Main path, part 2 (gather + score + label): one warp per query of the
// chunk, KA histogram slots per warp in shared memory.  Queries whose
// histogram does not fit are queued (chunk index) for the medium path.
template <int KA, int GB, class KeyT, class LocT>
__global__ void __launch_bounds__(CLS_WARPS * 32, 8) k_classify_score(ClassifyDb db, ClassifyQuery Q, uint32_t q0,
                                                                     uint32_t chunk, uint32_t list_cap,
                                                                     const uint64_t* __restrict__ glist,
                                                                     const uint4* __restrict__ meta,
                                                                     uint32_t* __restrict__ mid_list,
                                                                     uint32_t* __restrict__ mid_n) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    const size_t per_warp = scratch_bytes<uint16_t, KeyT>(KA, list_cap, 0, 0);
    const Scratch<uint16_t, KeyT> S = carve<uint16_t, KeyT>(smem + w * per_warp, KA, list_cap, 0, 0, WIN_A);
    Counters ctr;
    const uint32_t total = total_queries(Q);
    if (q0 >= total) return;
    const uint32_t nq = min(chunk, total - q0);
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarp = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < nq; i += nwarp) {
        const uint4 mt = meta[i];
        if (mt.x == ESCALATED) continue;
        // more locations than histogram slots: almost surely more distinct
        // locations than the histogram holds, so straight to the medium path
        if (mt.z > (uint32_t)KA) {
            if (lane == 0) mid_list[atomicAdd(mid_n, 1u)] = i;
            continue;
        }
        const uint64_t* src = glist + (uint64_t)i * list_cap;
        for (uint32_t j = lane; j < mt.x; j += 32) S.list[j] = __ldg(src + j);
        __syncwarp();
        const uint32_t q = q0 + i;
        if (query_score<GB, LocT>(db, Q, q, S, mt.x, meta_sws(mt), ctr) == Q_ESCALATE) {
            if (lane == 0) mid_list[atomicAdd(mid_n, 1u)] = i;
        } else {
            ctr.features += meta_feat(mt);
            ctr.found += mt.x;
            ctr.sectors += mt.w;
            ++ctr.queries;
        }
        __syncwarp();
    }
    flush_counters(Q, ctr, KC_SCORE);
}

// Queries of the chunk with h_lo < H <= h_hi gathered locations (h_lo = 0:
// no lower bound), not escalated: a warp takes groups of 32 consecutive
// queries from a counter (*ctr, zero before the launch), reads their
// metadata at once and takes those in range by ballot, so that warps that
// start late take fewer groups.  With mid_list, the queries beyond h_hi
// are queued there (chunk index) as they are met.
struct ChunkScan {
    uint32_t base, nq;  // first query of the current group, chunk size
    uint32_t* ctr;      // next group
    uint4 mt;           // this lane's query of the group
    uint32_t todo;      // lanes of the group still to be processed
};

__device__ __forceinline__ ChunkScan chunk_scan(uint32_t nq, uint32_t* ctr) {
    ChunkScan it;
    it.nq = nq;
    it.ctr = ctr;
    it.base = 0;
    it.todo = 0;
    return it;
}

__device__ __forceinline__ bool next_chunk_query(ChunkScan& it, const uint4* __restrict__ meta, uint32_t h_lo,
                                                uint32_t h_hi, uint32_t* __restrict__ mid_list,
                                                uint32_t* __restrict__ mid_n, uint32_t& i, uint4& mt) {
    const uint32_t lane = lane_id();
    while (it.todo == 0) {
        uint32_t g = 0;
        if (lane == 0) g = atomicAdd(it.ctr, 1u);
        g = __shfl_sync(FULL_MASK, g, 0);
        const uint64_t first = (uint64_t)g * 32;
        if (first >= it.nq) return false;
        it.base = (uint32_t)first;
        const uint64_t qi = first + lane;
        it.mt = qi < it.nq ? meta[qi] : make_uint4(ESCALATED, 0, 0, 0);
        const bool in = it.mt.x != ESCALATED && !(h_lo && it.mt.z <= h_lo);
        if (mid_list && in && it.mt.z > h_hi) mid_list[atomicAdd(mid_n, 1u)] = (uint32_t)qi;
        it.todo = __ballot_sync(FULL_MASK, in && it.mt.z <= h_hi);
    }
    const int l = __ffs(it.todo) - 1;
    it.todo &= it.todo - 1;
    i = it.base + (uint32_t)l;
    mt.x = __shfl_sync(FULL_MASK, it.mt.x, l);
    mt.y = __shfl_sync(FULL_MASK, it.mt.y, l);
    mt.z = __shfl_sync(FULL_MASK, it.mt.z, l);
    mt.w = __shfl_sync(FULL_MASK, it.mt.w, l);
    return true;
}

// One medium-path query (chunk index i): bucket list to working memory,
// hash-histogram scoring; a query that does not fit is queued for the
// large path.
template <int GB, class KeyT, class LocT>
__device__ __forceinline__ void medium_query(const ClassifyDb& db, const ClassifyQuery& Q, uint32_t q0,
                                             uint32_t list_cap, const uint64_t* __restrict__ glist,
                                             const Scratch<uint16_t, KeyT>& S, uint32_t i, const uint4& mt,
                                             uint32_t* __restrict__ ovf_list, uint32_t* __restrict__ ovf_n,
                                             Counters& ctr, unsigned long long& n_medium) {
    const uint32_t lane = lane_id();
    const uint64_t* src = glist + (uint64_t)i * list_cap;
    for (uint32_t j = lane; j < mt.x; j += 32) S.list[j] = __ldg(src + j);
    __syncwarp();
    const uint32_t q = q0 + i;
    if (query_score<GB, LocT>(db, Q, q, S, mt.x, meta_sws(mt), ctr) == Q_ESCALATE) {
        if (lane == 0) ovf_list[atomicAdd(ovf_n, 1u)] = q;
    } else {
        ctr.features += meta_feat(mt);
        ctr.found += mt.x;
        ctr.sectors += mt.w;
        ++ctr.queries;
        ++n_medium;
    }
    __syncwarp();
}

// Medium path: the queries queued by the hash path's score kernel or the
// sort path's largest size class, one warp each (work queue), KM_SLOTS
// histogram slots per warp in shared memory, the bucket list taken over
// from the lookup.  Queries that do not fit here either go to the large
// path.
template <int GB, class KeyT, class LocT>
__global__ void __launch_bounds__(MED_WARPS * 32) k_classify_medium(ClassifyDb db, ClassifyQuery Q, uint32_t q0,
                                                                   uint32_t list_cap,
                                                                   const uint64_t* __restrict__ glist,
                                                                   const uint4* __restrict__ meta,
                                                                   const uint32_t* __restrict__ mid_list,
                                                                   const uint32_t* __restrict__ mid_n,
                                                                   uint32_t* __restrict__ mid_work,
                                                                   uint32_t* __restrict__ ovf_list,
                                                                   uint32_t* __restrict__ ovf_n) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5;
    const uint32_t lane = lane_id();
    const size_t per_warp = scratch_bytes<uint16_t, KeyT>(KM_SLOTS, list_cap, 0, 0);
    const Scratch<uint16_t, KeyT> S = carve<uint16_t, KeyT>(smem + w * per_warp, KM_SLOTS, list_cap, 0, 0, WIN_A);
    Counters ctr;
    unsigned long long n_medium = 0;
    // a kernel launched after this one with programmatic stream
    // serialization (a sort-path class, which shares no data with this one)
    // may start while this one's few long queries finish
    asm volatile("griddepcontrol.launch_dependents;");
    const uint32_t n = *mid_n;
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(mid_work, 1u);
        k = __shfl_sync(FULL_MASK, k, 0);
        if (k >= n) break;
        const uint32_t i = mid_list[k];
        medium_query<GB, KeyT, LocT>(db, Q, q0, list_cap, glist, S, i, meta[i], ovf_list, ovf_n, ctr, n_medium);
    }
    flush_counters(Q, ctr, KC_MEDIUM);
    if (Q.counters && lane == 0 && n_medium) atomicAdd(Q.counters + 6, n_medium);
}

// ------------------------------------------------------------------
// Sort path (databases with 32-bit locations): query steps 5-8 of
// Section 5.2 for a query of at most 32*E gathered locations, on one warp,
// by sorting instead of hashing.  The paper compacts the gathered locations
// and sorts each read's segment (Sections 5.4-5.5); here one warp gathers
// the query's locations straight into registers (E per lane, all loads in
// flight at once), sorts them with an in-register bitonic network, and
// reads off the window count statistic (runs of equal locations) and the
// sliding-window scores (Section 5.6: elements in [x, x + sws) of the sorted
// array) without a hash table.  Same outputs as query_score.

// Bitonic sort of 32*E keys held E per lane, element i = lane*E + r, into
// ascending order of i.  Mirror form of the network: each merge stage of
// block size K starts by comparing i with its mirror i ^ (K - 1) and goes on
// with half-cleaners i ^ J, J = K/4 .. 1, and every comparator puts the
// smaller key at the smaller index, so the steps within a lane's registers
// need no direction select.  Stages up to K = E stay in the lane's
// registers; the stages beyond run as a loop whose body holds one mirror
// step, the cross-lane half-cleaners (each guarded by the stage) and the
// E/2 .. 1 in-register half-cleaners, which keeps the code small.
template <int E>
__device__ __forceinline__ void sort_in_lane_halves(uint32_t (&k)[E]) {
#pragma unroll
    for (int J = E >> 1; J > 0; J >>= 1) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if ((r & J) == 0) {
                const uint32_t a = k[r], b = k[r | J];
                k[r] = min(a, b);
                k[r | J] = max(a, b);
            }
        }
    }
}

template <int E>
__device__ __forceinline__ void warp_bitonic_sort(uint32_t (&k)[E]) {
    const uint32_t lane = lane_id();
#pragma unroll
    for (int K = 2; K <= E; K <<= 1) {
#pragma unroll
        for (int r = 0; r < E; ++r) {
            if ((r & (K >> 1)) == 0) {
                const int o = r ^ (K - 1);
                const uint32_t a = k[r], b = k[o];
                k[r] = min(a, b);
                k[o] = max(a, b);
            }
        }
#pragma unroll
        for (int J = K >> 2; J > 0; J >>= 1) {
#pragma unroll
            for (int r = 0; r < E; ++r) {
                if ((r & J) == 0) {
                    const uint32_t a = k[r], b = k[r | J];
                    k[r] = min(a, b);
                    k[r | J] = max(a, b);
                }
            }
        }
    }
#pragma unroll 1
    for (uint32_t kl = 2; kl <= 32; kl <<= 1) {  // K = kl * E
        {
            // mirror partner of element (lane, r): lane ^ (kl - 1), register
            // E-1-r; the lower lane keeps the minimum.  As a mirror pair
            // (r, E-1-r) of this lane meets the pair (E-1-r, r) of the
            // partner, each register takes the partner's value first.
            const uint32_t up = (lane & (kl >> 1)) ? 0xFFFFFFFFu : 0u;  // the upper lane keeps the max
            const uint32_t lm = kl - 1;
#pragma unroll
            for (int r = 0; r < E / 2; ++r) {
                const uint32_t a = k[r], b = k[E - 1 - r];
                const uint32_t pa = __shfl_xor_sync(FULL_MASK, b, lm);  // partner's E-1-r
                const uint32_t pb = __shfl_xor_sync(FULL_MASK, a, lm);  // partner's r
                const uint32_t na = min(a, pa), nb = min(b, pb);
                k[r] = na ^ ((na ^ max(a, pa)) & up);
                k[E - 1 - r] = nb ^ ((nb ^ max(b, pb)) & up);
            }
        }
#pragma unroll
        for (int t = 3; t >= 0; --t) {  // lane distances kl/4 .. 1 (warp-uniform guard)
            const uint32_t lj = 1u << t;
            if (lj <= (kl >> 2)) {
                const uint32_t up = (lane & lj) ? 0xFFFFFFFFu : 0u;
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const uint32_t o = __shfl_xor_sync(FULL_MASK, k[r], lj);
                    const uint32_t n = min(k[r], o);
                    k[r] = n ^ ((n ^ max(k[r], o)) & up);
                }
            }
        }
        sort_in_lane_halves<E>(k);
    }
}

// Per-warp shared memory of the sort path: bucket list, its prefix, and per
// run of equal locations in the sorted gather (at most 32*E runs) its
// location, its first sorted index and its score.
template <int E>
__host__ __device__ constexpr size_t sort_warp_bytes(uint32_t list_cap) {
    return align16((size_t)list_cap * 8) + align16(((size_t)list_cap + 4) * 4) + align16((32 * (size_t)E + 4) * 4) +
           align16((32 * (size_t)E + 4) * 2) + align16((32 * (size_t)E) * 2);
}

// Slot of loc[] and rs[] beyond every run (the arrays hold 32*E + 4).
template <int E>
constexpr uint32_t SORT_SPARE_SLOT = 32 * E + 3;

struct SortWarpMem {
    uint64_t* list;   // found buckets, offset << 16 | size
    uint32_t* l_pre;  // exclusive prefix of the bucket sizes
    uint32_t* loc;    // location of run j, ascending
    uint16_t* rs;     // first sorted index of run j; rs[D] = H
    uint16_t* sc;     // sliding-window score of run j (0 once excluded)
};

template <int E>
__device__ __forceinline__ SortWarpMem sort_warp_mem(unsigned char* p, uint32_t list_cap) {
    SortWarpMem m;
    m.list = reinterpret_cast<uint64_t*>(p);
    p += align16((size_t)list_cap * 8);
    m.l_pre = reinterpret_cast<uint32_t*>(p);
    p += align16(((size_t)list_cap + 4) * 4);
    m.loc = reinterpret_cast<uint32_t*>(p);
    p += align16((32 * (size_t)E + 4) * 4);
    m.rs = reinterpret_cast<uint16_t*>(p);
    p += align16((32 * (size_t)E + 4) * 2);
    m.sc = reinterpret_cast<uint16_t*>(p);
    return m;
}

constexpr int SORT_WARPS = 4;  // warps per CTA of the sort path

// First run index in [lo, hi) whose location is greater than v (hi if none).
__device__ __forceinline__ uint32_t runs_upper_bound(const uint32_t* loc, uint32_t lo, uint32_t hi, uint32_t v) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (loc[mid] <= v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Sort path, step 1 of a query: copies its bucket list from src to working
// memory and issues the loads of its H <= 32*E locations into k (element
// x = r * 32 + lane of the flat location list; NO_LOC beyond H).
constexpr uint32_t NO_LOC = 0xFFFFFFFFu;  // padding; sorts last and lies beyond H

template <int E>
__device__ __forceinline__ void sort_gather(const ClassifyDb& db, const SortWarpMem& M, const uint64_t* src,
                                           uint32_t n_list, uint32_t H, uint32_t (&k)[E]) {
    const uint32_t lane = lane_id();
    const uint32_t* __restrict__ locs = static_cast<const uint32_t*>(db.locs);
    uint64_t* list = M.list;
    uint32_t* l_pre = M.l_pre;
    __syncwarp();  // the previous query is done with the list
    for (uint32_t j = lane; j < n_list; j += 32) list[j] = __ldg(src + j);
    __syncwarp();

    // exclusive prefix of the bucket sizes
    uint32_t tot = 0;
    for (uint32_t base = 0; base < n_list; base += 32) {
        const uint32_t idx = base + lane;
        const uint32_t c = idx < n_list ? (uint32_t)(list[idx] & 0xFFFFu) : 0;
        uint32_t inc = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t x = __shfl_up_sync(FULL_MASK, inc, d);
            if ((int)lane >= d) inc += x;
        }
        if (idx < n_list) l_pre[idx] = tot + inc - c;
        tot += __shfl_sync(FULL_MASK, inc, 31);
    }
    if (lane == 0) l_pre[n_list] = tot;
    __syncwarp();

    uint32_t lo = 0, hi = n_list;  // bucket of x = lane: last b with l_pre[b] <= lane
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (l_pre[mid] <= lane) lo = mid; else hi = mid;
    }
    uint32_t bkt = lo;
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const uint32_t x = (uint32_t)r * 32 + lane;
        k[r] = NO_LOC;
        if (x < H) {
            while (l_pre[bkt + 1] <= x) ++bkt;
            k[r] = __ldg(locs + (list[bkt] >> 16) + (x - l_pre[bkt]));
        }
    }
}

// Sort path, step 2 of a query: its H gathered locations k (as left by
// sort_gather) are sorted, scored and labelled, and the outputs written.
template <int E>
__device__ __forceinline__ void query_sort(const ClassifyDb& db, const ClassifyQuery& Q, uint32_t q,
                                          const SortWarpMem& M, uint32_t sws, uint32_t H, uint32_t (&k)[E],
                                          Counters& ctr) {
    const uint32_t lane = lane_id();
    const uint32_t jb = db.jbits;
    warp_bitonic_sort<E>(k);

    // Runs of equal locations (the window count statistic of Section 5.6):
    // run j has location loc[j] and covers sorted indices [rs[j], rs[j+1]).
    uint32_t D;
    {
        // bit r of starts: element lane*E + r (< H) begins a run
        using Mask = typename std::conditional<(E > 32), unsigned long long, uint32_t>::type;
        constexpr int MB = 8 * (int)sizeof(Mask);
        const uint32_t before = __shfl_up_sync(FULL_MASK, k[E - 1], 1);
        Mask starts = 0;
#pragma unroll
        for (int r = 0; r < E; ++r) starts |= (Mask)(k[r] != (r ? k[r - 1] : before)) << r;
        const uint32_t first = lane * E;
        const uint32_t valid = H > first ? min((uint32_t)E, H - first) : 0u;
        starts &= valid >= (uint32_t)MB ? ~(Mask)0 : (((Mask)1 << valid) - 1);
        if (lane == 0 && H > 0) starts |= 1;
        const uint32_t n = (uint32_t)(MB == 64 ? __popcll((unsigned long long)starts) : __popc((uint32_t)starts));
        uint32_t inc = n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t x = __shfl_up_sync(FULL_MASK, inc, d);
            if ((int)lane >= d) inc += x;
        }
        D = __shfl_sync(FULL_MASK, inc, 31);
        // the run starts in order (for E = 32 the other elements write to a
        // spare slot instead of being predicated off, which keeps the
        // kernel's predicate registers within what the compiler can allocate)
        uint32_t pos = inc - n;
#pragma unroll
        for (int r = 0; r < E; ++r) {
            const uint32_t b = (uint32_t)(starts >> r) & 1u;
            if (E >= 32) {
                const uint32_t at = b ? pos : SORT_SPARE_SLOT<E>;
                M.loc[at] = k[r];
                M.rs[at] = (uint16_t)(lane * E + r);
            } else if (b) {
                M.loc[pos] = k[r];
                M.rs[pos] = (uint16_t)(lane * E + r);
            }
            pos += b;
        }
        __syncwarp();
        if (lane == 0) M.rs[D] = (uint16_t)H;
    }
    __syncwarp();
    ctr.locations += H;
    ctr.distinct += D;

    // Sliding-window scores (Section 5.6): the score of run j is the number
    // of sorted locations in [loc[j], hi], hi = loc[j] + sws - 1 cut at the
    // last window id of the target.  Runs have distinct locations, so at most
    // sws - 1 runs after j lie in that range; e is the first run beyond it
    // and the score is rs[e] - rs[j].  Four runs are checked per step (the
    // locations ascend, so the count of those <= hi is the advance).  The
    // first top-m round is folded in.
    const uint32_t jmask = (1u << jb) - 1u;
    const uint32_t w1 = sws ? sws - 1 : 0u;  // no wrap: stays in the run's target
    Cand best = Cand{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0};
    for (uint32_t j = lane; j < D; j += 32) {
        const uint32_t x = M.loc[j];
        const uint32_t hi = x + min(w1, jmask - (x & jmask));
        uint32_t e = j + 1;
        for (;;) {
            uint32_t adv = 0;
#pragma unroll
            for (int d = 0; d < 4; ++d) adv += (e + d < D && M.loc[e + d] <= hi) ? 1u : 0u;
            e += adv;
            if (adv < 4) break;
        }
        const uint32_t sc = (uint32_t)M.rs[e] - (uint32_t)M.rs[j];
        M.sc[j] = (uint16_t)sc;
        const Cand c = Cand{sc, x >> jb, x & jmask, 0};
        if (better(c, best)) best = c;
    }
    __syncwarp();

    // top m with one candidate per target (Section 4.2 / 5.6): rounds of
    // warp arg-max; the winner's target is excluded from later rounds by
    // zeroing the scores of its runs; the label is folded as in
    // query_score.  Unless the full top-m list is requested, later rounds
    // only matter for "close" candidates, so after the first round every
    // score below the close threshold is cleared at once.
    const int m = (int)Q.m;
    Cand mine = Cand{0, 0xFFFFFFFFu, 0, 0};
    uint32_t label = NO_TAXON, hits = 0, top = 0xFFFFFFFFu;
    uint64_t bar = 0;
    uint32_t prev_t = 0xFFFFFFFFu;
    for (int rd = 0; rd < m; ++rd) {
        if (rd) {
            best = Cand{0, 0xFFFFFFFFu, 0xFFFFFFFFu, 0};
            for (uint32_t j = lane; j < D; j += 32) {
                const uint32_t sc = M.sc[j];
                if (sc == 0) continue;
                const uint32_t x = M.loc[j];
                const uint32_t t = x >> jb;
                if (t == prev_t) {
                    M.sc[j] = 0;
                    continue;
                }
                const Cand c = Cand{sc, t, x & jmask, 0};
                if (better(c, best)) best = c;
            }
        }
        {
            const uint32_t ms = __reduce_max_sync(FULL_MASK, best.score);
            const uint32_t mt = __reduce_min_sync(FULL_MASK, best.score == ms ? best.t : 0xFFFFFFFFu);
            const uint32_t mj =
                __reduce_min_sync(FULL_MASK, (best.score == ms && best.t == mt) ? best.j0 : 0xFFFFFFFFu);
            best = Cand{ms, mt, mj, 0};
        }
        if (best.score == 0) break;
        prev_t = best.t;
        if (Q.cands) {
            // last window of the range present: the location of the last run <= hi
            const uint32_t x0 = (best.t << jb) | best.j0;
            const uint32_t hi = x0 + min(w1, jmask - best.j0);
            const uint32_t e = runs_upper_bound(M.loc, 0, D, hi);
            best.j1 = M.loc[e - 1] & jmask;
        }
        if ((int)lane == rd) mine = best;
        if (rd == 0) {
            hits = best.score;
            top = best.t;
            bar = (uint64_t)(100 - Q.band) * hits;
            if (hits >= Q.hits_min) label = top < db.n_targets ? db.taxon_of_target[top] : NO_TAXON;
            else if (!Q.cands) break;
            if (!Q.cands) {
                // smallest score s with 100 s >= bar
                const uint32_t s_min = (uint32_t)((bar + 99) / 100);
                for (uint32_t j = lane; j < D; j += 32)
                    if (M.sc[j] < s_min) M.sc[j] = 0;
            }
        } else if (hits >= Q.hits_min && 100ull * best.score >= bar) {
            const uint32_t tx = best.t < db.n_targets ? db.taxon_of_target[best.t] : NO_TAXON;
            label = lca2(db, label, tx);
        } else if (!Q.cands) {
            break;
        }
        __syncwarp();
    }
    write_result(Q, q, label, hits, top, mine);
}

// Resident CTAs per SM that the register budget of a sort-path kernel is
// sized for (shared memory admits 15, 10, 5 and 3 for E = 8, 16, 32, 64).
template <int E>
constexpr int sort_min_ctas() { return E == 8 ? 8 : (E == 16 ? 7 : (E == 32 ? 5 : 3)); }

// Sort path over the chunk's queries with h_lo < H <= 32*E gathered
// locations; with mid_list (the largest class), larger ones are queued for
// the medium path.
template <int E>
__global__ void __launch_bounds__(SORT_WARPS * 32, sort_min_ctas<E>()) k_classify_sort(ClassifyDb db, ClassifyQuery Q, uint32_t q0,
                                                                  uint32_t chunk, uint32_t list_cap,
                                                                  const uint64_t* __restrict__ glist,
                                                                  const uint4* __restrict__ meta, uint32_t h_lo,
                                                                  uint32_t* __restrict__ mid_list,
                                                                  uint32_t* __restrict__ mid_n,
                                                                  uint32_t* __restrict__ group_ctr) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t w = threadIdx.x >> 5;
    const SortWarpMem M = sort_warp_mem<E>(smem + w * sort_warp_bytes<E>(list_cap), list_cap);
    Counters ctr;
    const uint32_t total = total_queries(Q);
    if (q0 < total) {
        ChunkScan it = chunk_scan(min(chunk, total - q0), group_ctr);
        uint32_t i;
        uint4 mt;
        uint32_t k[E];
        while (next_chunk_query(it, meta, h_lo, 32u * E, mid_list, mid_n, i, mt)) {
            sort_gather<E>(db, M, glist + (uint64_t)i * list_cap, mt.x, mt.z, k);
            query_sort<E>(db, Q, q0 + i, M, meta_sws(mt), mt.z, k, ctr);
            ctr.features += meta_feat(mt);
            ctr.found += mt.x;
            ctr.sectors += mt.w;
            ++ctr.queries;
        }
        flush_counters(Q, ctr, E == 8 ? 1 : (E == 16 ? 2 : (E == 32 ? 3 : 6)));
    }
    // Launched as a programmatic dependent of the medium path, this kernel
    // may run alongside it; waiting for that grid before exiting makes this
    // kernel's completion imply the medium path's, so that later work in
    // the stream or graph never overtakes it.  A no-op for an ordinary
    // launch.
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Large path: queries queued by the shared-memory path, one warp each, with
// working memory in global scratch.
template <int R, int KC, class LocT>
__global__ void __launch_bounds__(CLS_WARPS * 32, 4) k_classify_large(ClassifyDb db, ClassifyQuery Q,
                                                                   const uint32_t* __restrict__ ovf_list,
                                                                   const uint32_t* __restrict__ ovf_n,
                                                                   uint32_t* __restrict__ work,
                                                                   unsigned char* __restrict__ scratch,
                                                                   size_t per_warp) {
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const Scratch<uint32_t> S =
        carve<uint32_t>(scratch + gw * per_warp, KB_SLOTS, LIST_B, LIST_B, BUF_B, MC_MAX_QUERY_WINDOWS);
    Counters ctr;
    const uint32_t n = *ovf_n;
    unsigned long long n_large = 0;
    for (;;) {
        uint32_t i = 0;
        if (lane_id() == 0) i = atomicAdd(work, 1u);
        i = __shfl_sync(FULL_MASK, i, 0);
        if (i >= n) break;
        const uint32_t q = ovf_list[i];
        ++n_large;
        int r = process_query<R, KC, LocT>(db, Q, q, S, ctr);
        if (r != Q_DONE) {
            write_unclassified(Q, q);
            if (lane_id() == 0) atomicMax(Q.status, DEV_ERR_CAPACITY);
        }
        __syncwarp();
    }
    flush_counters(Q, ctr, KC_LARGE);
    if (Q.counters && lane_id() == 0 && n_large) atomicAdd(Q.counters + 3, n_large);
}


constexpr uint32_t CHUNK = CLASSIFY_CHUNK;

using LookupKernel = void (*)(ClassifyDb, ClassifyQuery, uint32_t, uint32_t, uint32_t, uint64_t*, uint4*, uint32_t*,
                              uint32_t*);
using ScoreKernel = void (*)(ClassifyDb, ClassifyQuery, uint32_t, uint32_t, uint32_t, const uint64_t*, const uint4*,
                             uint32_t*, uint32_t*);
using LargeKernel = void (*)(ClassifyDb, ClassifyQuery, const uint32_t*, const uint32_t*, uint32_t*, unsigned char*,
                             size_t);
using MediumKernel = void (*)(ClassifyDb, ClassifyQuery, uint32_t, uint32_t, const uint64_t*, const uint4*,
                              const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint32_t*);

template <int R, int KC>
LookupKernel lookup_for_lb(uint32_t lb) {
    if (lb == 2) return k_classify_lookup<R, KC, 2>;
    if (lb == 8) return k_classify_lookup<R, KC, 8>;
    return k_classify_lookup<R, KC, 4>;
}

LookupKernel pick_lookup(const SketchParams& sp, uint32_t lb) {
    const int r = sketch_r_for(sp.w);
    const bool k16 = sp.k == 16;
    if (r == 4) return k16 ? lookup_for_lb<4, 16>(lb) : lookup_for_lb<4, 0>(lb);
    if (r == 8) return k16 ? lookup_for_lb<8, 16>(lb) : lookup_for_lb<8, 0>(lb);
    return k16 ? lookup_for_lb<16, 16>(lb) : lookup_for_lb<16, 0>(lb);
}

template <int KA, class KeyT, class LocT>
ScoreKernel score_for_gb(uint32_t gb) {
    if (gb == 4) return k_classify_score<KA, 4, KeyT, LocT>;
    if (gb == 16) return k_classify_score<KA, 16, KeyT, LocT>;
    return k_classify_score<KA, 8, KeyT, LocT>;
}

template <class KeyT, class LocT>
ScoreKernel score_for_ka(uint32_t ka, uint32_t gb) {
    if (ka == 256) return score_for_gb<256, KeyT, LocT>(gb);
    if (ka == 1024) return score_for_gb<1024, KeyT, LocT>(gb);
    return score_for_gb<512, KeyT, LocT>(gb);
}

// Histogram key / location types of a launch: compact = 32-bit keys of
// 32-bit locations; wide = 64-bit keys of 32-bit locations; otherwise both
// 64-bit.
enum class KeyMode { compact, wide32, wide64 };

KeyMode key_mode(const ClassifyDb& db, const Tuning& t) {
    if (!db.jbits) return KeyMode::wide64;
    return t.wide_keys ? KeyMode::wide32 : KeyMode::compact;
}

ScoreKernel pick_score(uint32_t ka, uint32_t gb, KeyMode km) {
    if (km == KeyMode::compact) return score_for_ka<uint32_t, uint32_t>(ka, gb);
    if (km == KeyMode::wide32) return score_for_ka<uint64_t, uint32_t>(ka, gb);
    return score_for_ka<uint64_t, uint64_t>(ka, gb);
}

MediumKernel pick_medium(KeyMode km) {
    if (km == KeyMode::compact) return k_classify_medium<GB_DEFAULT, uint32_t, uint32_t>;
    if (km == KeyMode::wide32) return k_classify_medium<GB_DEFAULT, uint64_t, uint32_t>;
    return k_classify_medium<GB_DEFAULT, uint64_t, uint64_t>;
}

template <class LocT>
LargeKernel pick_large_t(const SketchParams& sp) {
    const int r = sketch_r_for(sp.w);
    const bool k16 = sp.k == 16;
    if (r == 4) return k16 ? k_classify_large<4, 16, LocT> : k_classify_large<4, 0, LocT>;
    if (r == 8) return k16 ? k_classify_large<8, 16, LocT> : k_classify_large<8, 0, LocT>;
    return k16 ? k_classify_large<16, 16, LocT> : k_classify_large<16, 0, LocT>;
}

LargeKernel pick_large(const ClassifyDb& db) {
    return db.jbits ? pick_large_t<uint32_t>(db.sp) : pick_large_t<uint64_t>(db.sp);
}

// Kernels and launch shapes of one launch set.
using SortKernel = void (*)(ClassifyDb, ClassifyQuery, uint32_t, uint32_t, uint32_t, const uint64_t*, const uint4*,
                            uint32_t, uint32_t*, uint32_t*, uint32_t*);

// The sort path's size classes: queries of up to 256, 512, 1024 and 2048
// gathered locations, each with its own kernel (E = 8, 16, 32, 64 per lane).
constexpr int N_SORT_CLASSES = 4;
constexpr uint32_t SORT_CLASS_MAX[N_SORT_CLASSES] = {256, 512, 1024, 2048};

struct Geometry {
    LookupKernel kl;
    ScoreKernel ks;
    MediumKernel km;
    LargeKernel kb;
    SortKernel kt[N_SORT_CLASSES];
    bool sort;           // score by the sort path (else the hash path)
    int n_sort;          // sort classes in use
    uint32_t list_cap;
    size_t smem_l, smem_s, smem_m, per_warp_b, smem_t[N_SORT_CLASSES];
    uint32_t threads_l, threads_s, grid_l, grid_s, grid_m, blocks_b, grid_t[N_SORT_CLASSES];
};

cudaError_t geometry(const ClassifyDb& db, const Tuning& t, const ClassifyScratch& sc, Geometry* g) {
    cudaError_t e;
    int dev = 0, sms = NUM_SMS_HINT;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    g->list_cap = WIN_A * db.sp.s;
    g->kl = pick_lookup(db.sp, t.probe_batch);
    const KeyMode km = key_mode(db, t);
    const bool compact = km == KeyMode::compact;
    g->ks = pick_score(t.hist_slots, t.gather_batch, km);
    g->kb = pick_large(db);
    g->km = pick_medium(km);
    g->smem_m = MED_WARPS * (compact ? scratch_bytes<uint16_t, uint32_t>(KM_SLOTS, g->list_cap, 0, 0)
                                     : scratch_bytes<uint16_t, uint64_t>(KM_SLOTS, g->list_cap, 0, 0));
    if ((e = cudaFuncSetAttribute(g->km, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g->smem_m)) != cudaSuccess)
        return e;
    int occ_m = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_m, g->km, MED_WARPS * 32, g->smem_m)) != cudaSuccess)
        return e;
    g->grid_m = (uint32_t)sms * (uint32_t)std::max(occ_m, 1);
    g->threads_l = t.lookup_warps * 32;
    g->threads_s = t.score_warps * 32;
    g->smem_l = t.lookup_warps * lookup_warp_bytes(g->list_cap);
    g->smem_s = t.score_warps * (compact ? scratch_bytes<uint16_t, uint32_t>(t.hist_slots, g->list_cap, 0, 0)
                                         : scratch_bytes<uint16_t, uint64_t>(t.hist_slots, g->list_cap, 0, 0));
    if ((e = cudaFuncSetAttribute(g->kl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g->smem_l)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(g->ks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g->smem_s)) != cudaSuccess)
        return e;
    int occ_l = 1, occ_s = 1;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_l, g->kl, g->threads_l, g->smem_l)) != cudaSuccess)
        return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, g->ks, g->threads_s, g->smem_s)) != cudaSuccess)
        return e;
    occ_l = std::max(occ_l, 1);
    occ_s = std::max(occ_s, 1);
    const uint64_t c = std::max<uint32_t>(sc.chunk, 1);
    g->grid_l = (uint32_t)std::min<uint64_t>((c + t.lookup_warps - 1) / t.lookup_warps, (uint64_t)sms * occ_l);
    g->grid_s = (uint32_t)std::min<uint64_t>((c + t.score_warps - 1) / t.score_warps, (uint64_t)sms * occ_s);
    g->per_warp_b = scratch_bytes<uint32_t>(KB_SLOTS, LIST_B, LIST_B, BUF_B);
    g->blocks_b = std::max<uint32_t>(1, sc.large_warps / CLS_WARPS);
    // sort path: only for 32-bit locations with compact keys
    g->sort = compact && t.score_mode != SCORE_HASH;
    g->n_sort = 0;
    if (g->sort) {
        const SortKernel kts[N_SORT_CLASSES] = {k_classify_sort<8>, k_classify_sort<16>, k_classify_sort<32>,
                                                k_classify_sort<64>};
        const size_t bytes[N_SORT_CLASSES] = {sort_warp_bytes<8>(g->list_cap), sort_warp_bytes<16>(g->list_cap),
                                              sort_warp_bytes<32>(g->list_cap), sort_warp_bytes<64>(g->list_cap)};
        for (int c2 = 0; c2 < N_SORT_CLASSES && SORT_CLASS_MAX[c2] <= t.sort_max; ++c2) {
            g->kt[c2] = kts[c2];
            g->smem_t[c2] = SORT_WARPS * bytes[c2];
            if ((e = cudaFuncSetAttribute(kts[c2], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g->smem_t[c2])) !=
                cudaSuccess)
                return e;
            int occ_t = 1;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_t, kts[c2], SORT_WARPS * 32, g->smem_t[c2])) !=
                cudaSuccess)
                return e;
            g->grid_t[c2] = (uint32_t)std::min<uint64_t>((c + SORT_WARPS - 1) / SORT_WARPS,
                                                         (uint64_t)sms * std::max(occ_t, 1));
            g->n_sort = c2 + 1;
        }
    }
    return cudaSuccess;
}

__host__ __device__ constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch layout: escalation queue + counters, chunk metadata, medium-path
// queue, chunk bucket lists, large-path working memory.
struct ScratchLayout {
    size_t ovf, meta, mid, glist, large, total;
    uint32_t chunk;
};

constexpr ScratchLayout scratch_layout(uint32_t n_q_cap, uint32_t sketch_size, uint32_t large_warps) {
    ScratchLayout L{};
    const size_t list_cap = (size_t)WIN_A * sketch_size;
    const size_t per_warp_b = scratch_bytes<uint32_t>(KB_SLOTS, LIST_B, LIST_B, BUF_B);
    L.chunk = n_q_cap < CHUNK ? n_q_cap : CHUNK;
    L.ovf = 0;
    L.meta = align256(L.ovf + ((size_t)n_q_cap + 16) * 4);
    L.mid = align256(L.meta + (size_t)L.chunk * sizeof(uint4));
    L.glist = align256(L.mid + (size_t)L.chunk * 4);
    L.large = align256(L.glist + (size_t)L.chunk * list_cap * 8);
    L.total = align256(L.large + (size_t)large_warps * per_warp_b);
    return L;
}

// Queue counters: [0] large-path queue length, [1] large-path work counter,
// [2] medium-path queue length, [3] medium-path work counter, [4] saved
// large-path queue length (autotuner), [5 + c] group counter of sort-path
// class c.
uint32_t* queue_counters(const ClassifyScratch& sc) { return sc.ovf + sc.n_q_cap; }

cudaError_t launch_lookup(const Geometry& g, const ClassifyDb& db, const ClassifyQuery& Q, const ClassifyScratch& sc,
                          uint32_t q0, cudaStream_t s) {
    MC_LAUNCH("classify_lookup", s,
              g.kl<<<g.grid_l, g.threads_l, g.smem_l, s>>>(db, Q, q0, sc.chunk, g.list_cap, sc.glist, sc.meta, sc.ovf,
                                                          queue_counters(sc)));
    return cudaGetLastError();
}

// Medium path of the chunk at q0 (its queue).
cudaError_t launch_medium(const Geometry& g, const ClassifyDb& db, const ClassifyQuery& Q, const ClassifyScratch& sc,
                          uint32_t q0, cudaStream_t s) {
    uint32_t* qc = queue_counters(sc);
    MC_LAUNCH("classify_medium", s,
              g.km<<<g.grid_m, MED_WARPS * 32, g.smem_m, s>>>(db, Q, q0, g.list_cap, sc.glist, sc.meta, sc.mid, qc + 2,
                                                             qc + 3, sc.ovf, qc));
    return cudaGetLastError();
}

// Score of the chunk at q0.  Sort path: the largest size class first (it
// queues the queries beyond it), then the medium path, then the other
// classes, the most populous one (512) launched with programmatic stream
// serialization so that it fills the SMs the medium path's few long
// queries leave idle (they share no data: the sort kernels read the
// lookup's outputs and write other queries' results; their groups of
// queries come from a counter, so the CTAs that start late take fewer).
// Hash path: the score kernel, then the medium path for the queries whose
// histogram did not fit.
cudaError_t launch_score(const Geometry& g, const ClassifyDb& db, const ClassifyQuery& Q, const ClassifyScratch& sc,
                         uint32_t q0, cudaStream_t s) {
    uint32_t* qc = queue_counters(sc);
    cudaError_t e = cudaMemsetAsync(qc + 2, 0, 2 * sizeof(uint32_t), s);  // medium queue; [4] is kept
    if (e != cudaSuccess) return e;
    if (g.sort && (e = cudaMemsetAsync(qc + 5, 0, N_SORT_CLASSES * sizeof(uint32_t), s)) != cudaSuccess) return e;
    if (!g.sort) {
        MC_LAUNCH("classify_score", s,
                  g.ks<<<g.grid_s, g.threads_s, g.smem_s, s>>>(db, Q, q0, sc.chunk, g.list_cap, sc.glist, sc.meta,
                                                              sc.mid, qc + 2));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        return launch_medium(g, db, Q, sc, q0, s);
    }
    static const char* const names[N_SORT_CLASSES] = {"classify_sort256", "classify_sort512", "classify_sort1024",
                                                      "classify_sort2048"};
    const int last = g.n_sort - 1;
    const int pdl = last >= 2 ? 1 : -1;  // the class launched as the medium path's dependent
    int order[N_SORT_CLASSES + 1], n = 0;
    order[n++] = last;
    order[n++] = -1;  // medium path
    if (pdl >= 0) order[n++] = pdl;
    for (int c = 0; c < last; ++c)
        if (c != pdl) order[n++] = c;
    for (int k = 0; k < n; ++k) {
        const int c = order[k];
        if (c < 0) {
            if ((e = launch_medium(g, db, Q, sc, q0, s)) != cudaSuccess) return e;
            continue;
        }
        const uint32_t h_lo = c ? SORT_CLASS_MAX[c - 1] : 0;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g.grid_t[c]);
        cfg.blockDim = dim3(SORT_WARPS * 32);
        cfg.dynamicSmemBytes = g.smem_t[c];
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = c == pdl ? 1 : 0;
        uint32_t* ml = c == last ? sc.mid : nullptr;
        uint32_t* mn = c == last ? qc + 2 : nullptr;
        MC_LAUNCH(names[c], s,
                  e = cudaLaunchKernelEx(&cfg, g.kt[c], db, Q, q0, (uint32_t)sc.chunk, g.list_cap,
                                         (const uint64_t*)sc.glist, (const uint4*)sc.meta, h_lo, ml, mn, qc + 5 + c));
        if (e != cudaSuccess) return e;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_large(const Geometry& g, const ClassifyDb& db, const ClassifyQuery& Q, const ClassifyScratch& sc,
                         cudaStream_t s) {
    uint32_t* qc = queue_counters(sc);
    MC_LAUNCH("classify_large", s,
              g.kb<<<g.blocks_b, CLS_WARPS * 32, 0, s>>>(db, Q, sc.ovf, qc, qc + 1, sc.large, g.per_warp_b));
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------ shard merge
// Sharded classification (Section 4.2: with the database partitioned over
// GPUs, the top candidates of every partition are merged).  One thread per
// query merges the per-shard top-m lists into the global top m (score
// descending, global target ascending; a target lives in one shard, so no
// candidate spans lists) and labels it as query_score does.
namespace {
__global__ void k_merge_candidates(ClassifyDb db, const uint32_t* __restrict__ taxon, uint32_t n_targets,
                                   const MergeList* __restrict__ lists, uint32_t n_lists, uint32_t n_q, uint32_t m,
                                   uint32_t hits_min, uint32_t band, uint32_t* __restrict__ label,
                                   uint32_t* __restrict__ hits, uint32_t* __restrict__ top_target,
                                   uint32_t* __restrict__ cands_out) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n_q; q += gridDim.x * blockDim.x) {
        uint32_t ts[MAX_M], tt[MAX_M], tj0[MAX_M], tj1[MAX_M];
#pragma unroll
        for (int a = 0; a < MAX_M; ++a) {
            ts[a] = 0;
            tt[a] = 0xFFFFFFFFu;
            tj0[a] = tj1[a] = 0;
        }
        for (uint32_t l = 0; l < n_lists; ++l) {
            const MergeList L = lists[l];
            for (uint32_t i = 0; i < m; ++i) {
                const uint4 c = *reinterpret_cast<const uint4*>(L.cands + ((uint64_t)q * m + i) * 4);
                if (c.x == 0) break;  // the rest of this list is empty
                uint32_t cs = c.x, ct = L.base + c.y, c0 = c.z, c1 = c.w;
                // one bubbling insertion pass (score descending, target ascending)
#pragma unroll
                for (int a = 0; a < MAX_M; ++a) {
                    if ((uint32_t)a < m && (cs > ts[a] || (cs == ts[a] && ct < tt[a]))) {
                        const uint32_t xs = ts[a], xt = tt[a], x0 = tj0[a], x1 = tj1[a];
                        ts[a] = cs;
                        tt[a] = ct;
                        tj0[a] = c0;
                        tj1[a] = c1;
                        cs = xs;
                        ct = xt;
                        c0 = x0;
                        c1 = x1;
                    }
                }
            }
        }
        uint32_t lab = NO_TAXON;
        const uint32_t h = ts[0];
        if (h > 0 && h >= hits_min) {
            lab = tt[0] < n_targets ? taxon[tt[0]] : NO_TAXON;
            const uint64_t bar = (uint64_t)(100 - band) * h;
#pragma unroll
            for (int a = 1; a < MAX_M; ++a) {
                if ((uint32_t)a >= m || ts[a] == 0 || 100ull * ts[a] < bar) break;
                lab = lca2(db, lab, tt[a] < n_targets ? taxon[tt[a]] : NO_TAXON);
            }
        }
        label[q] = lab;
        hits[q] = h;
        if (top_target) top_target[q] = h ? tt[0] : 0xFFFFFFFFu;
        if (cands_out) {
#pragma unroll
            for (int a = 0; a < MAX_M; ++a)
                if ((uint32_t)a < m)
                    *reinterpret_cast<uint4*>(cands_out + ((uint64_t)q * m + a) * 4) =
                        make_uint4(ts[a], ts[a] ? tt[a] : 0xFFFFFFFFu, ts[a] ? tj0[a] : 0, ts[a] ? tj1[a] : 0);
        }
    }
}
}  // namespace

cudaError_t merge_candidates(const Mem& mem, const ClassifyDb& db, const uint32_t* taxon, uint32_t n_targets,
                             const MergeList* lists, uint32_t n_lists, uint32_t n_q, uint32_t m, uint32_t hits_min,
                             uint32_t band, uint32_t* label, uint32_t* hits, uint32_t* top_target, uint32_t* cands_out,
                             cudaStream_t s) {
    if (n_q == 0) return cudaSuccess;
    Tmp<MergeList> dl(mem, std::max<uint32_t>(n_lists, 1), s);
    if (!dl.ok()) return cudaErrorMemoryAllocation;
    cudaError_t e;
    if (n_lists &&
        (e = cudaMemcpyAsync(dl.ptr, lists, n_lists * sizeof(MergeList), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n_q + 255) / 256, (uint64_t)NUM_SMS_HINT * 8);
    MC_LAUNCH("merge_candidates", s,
              k_merge_candidates<<<grid, 256, 0, s>>>(db, taxon, n_targets, dl.ptr, n_lists, n_q, m, hits_min, band,
                                                      label, hits, top_target, cands_out));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the host list array is read by the copy above: wait for it before returning
    return cudaStreamSynchronize(s);
}

uint32_t compact_key_bits(uint64_t n_targets, uint64_t max_windows) {
    auto bits = [](uint64_t x) { return x ? 64u - (uint32_t)__builtin_clzll(x) : 0u; };
    if (n_targets == 0 || max_windows == 0) return 0;
    const uint32_t jb = std::max(1u, bits(max_windows - 1));
    const uint32_t tb = bits(n_targets - 1);
    if (jb >= 32) return 0;  // one target of more than 2^31 windows: 64-bit locations
    if (jb + tb < 32) return jb;
    // 32 bits: usable unless the all-ones key (the empty-slot marker) is a
    // location; a sliding-window lookup of that key only ever meets empty
    // slots and counts 0
    if (jb + tb == 32 && !(n_targets == (1ull << tb) && max_windows == (1ull << jb))) return jb;
    return 0;
}

bool tuning_valid(const Tuning& t) {
    auto in = [](uint32_t v, std::initializer_list<uint32_t> set) {
        for (uint32_t x : set)
            if (v == x) return true;
        return false;
    };
    return in(t.hist_slots, {256, 512, 1024}) && in(t.probe_batch, {2, 4, 8}) && in(t.gather_batch, {4, 8, 16}) &&
           in(t.lookup_warps, {4, 8}) && in(t.score_warps, {2, 4}) && t.wide_keys <= 1 &&
           in(t.score_mode, {SCORE_SORT, SCORE_HASH}) && in(t.sort_max, {256, 512, 1024, 2048});
}

uint32_t classify_default_large_warps() {
    int dev = 0, sms = NUM_SMS_HINT;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = NUM_SMS_HINT;
    }
    return (uint32_t)std::max(CLS_WARPS, (sms * B_WARPS_PER_SM / CLS_WARPS) * CLS_WARPS);
}

size_t classify_scratch_bytes(uint32_t n_q_cap, uint32_t sketch_size, uint32_t large_warps) {
    return scratch_layout(n_q_cap, sketch_size, large_warps).total;
}

ClassifyScratch classify_scratch_carve(unsigned char* base, uint32_t n_q_cap, uint32_t sketch_size,
                                       uint32_t large_warps) {
    const ScratchLayout L = scratch_layout(n_q_cap, sketch_size, large_warps);
    ClassifyScratch sc;
    sc.ovf = reinterpret_cast<uint32_t*>(base + L.ovf);
    sc.meta = reinterpret_cast<uint4*>(base + L.meta);
    sc.mid = reinterpret_cast<uint32_t*>(base + L.mid);
    sc.glist = reinterpret_cast<uint64_t*>(base + L.glist);
    sc.large = base + L.large;
    sc.n_q_cap = n_q_cap;
    sc.chunk = L.chunk;
    sc.large_warps = large_warps;
    return sc;
}

cudaError_t classify_enqueue(const ClassifyDb& db, const ClassifyQuery& Q, const Tuning& t, const ClassifyScratch& sc,
                             cudaStream_t s, int* n_kernels) {
    cudaError_t e;
    int n = 0;
    if (n_kernels) *n_kernels = 0;
    if (Q.n_q == 0) return cudaSuccess;
    if (Q.n_q > sc.n_q_cap) return cudaErrorInvalidValue;
    Geometry g;
    if ((e = geometry(db, t, sc, &g)) != cudaSuccess) return e;
    // only the queue counters must start at zero
    if ((e = cudaMemsetAsync(queue_counters(sc), 0, 2 * sizeof(uint32_t), s)) != cudaSuccess) return e;
    for (uint32_t q0 = 0; q0 < Q.n_q; q0 += sc.chunk) {
        if ((e = launch_lookup(g, db, Q, sc, q0, s)) != cudaSuccess) return e;
        if ((e = launch_score(g, db, Q, sc, q0, s)) != cudaSuccess) return e;
        n += 2 + (g.sort ? g.n_sort : 1);
        if (sc.chunk == 0) break;
    }
    if ((e = launch_large(g, db, Q, sc, s)) != cudaSuccess) return e;
    if (n_kernels) *n_kernels = n + 1;
    return cudaSuccess;
}

cudaError_t classify_launch(const Mem& mem, const ClassifyDb& db, const ClassifyQuery& Q, const Tuning& t,
                            cudaStream_t s) {
    if (Q.n_q == 0) return cudaSuccess;
    const uint32_t lw = classify_default_large_warps();
    Tmp<unsigned char> buf(mem, classify_scratch_bytes(Q.n_q, db.sp.s, lw), s);
    if (!buf.ok()) return cudaErrorMemoryAllocation;
    const ClassifyScratch sc = classify_scratch_carve(buf.ptr, Q.n_q, db.sp.s, lw);
    return classify_enqueue(db, Q, t, sc, s, nullptr);
}

// Number of large-path warps of the allocation-free launch.
constexpr uint32_t NOALLOC_LARGE_WARPS = 8;
// The documented per-call maximum of the allocation-free entry point must
// fit its fixed scratch array at the largest sketch size.
static_assert(scratch_layout(MC_NOALLOC_MAX_QUERIES, MC_MAX_SKETCH, NOALLOC_LARGE_WARPS).total <=
                  MC_NOALLOC_SCRATCH_BYTES,
              "MC_NOALLOC_MAX_QUERIES queries at MC_MAX_SKETCH do not fit MC_NOALLOC_SCRATCH_BYTES");

size_t classify_noalloc_bytes(uint32_t n_q, uint32_t sketch_size) {
    return classify_scratch_bytes(n_q, sketch_size, NOALLOC_LARGE_WARPS);
}

cudaError_t classify_launch_noalloc(const ClassifyDb& db, const ClassifyQuery& Q, const Tuning& t,
                                   unsigned char* scratch, size_t scratch_len, cudaStream_t s) {
    if (Q.n_q == 0) return cudaSuccess;
    if (classify_noalloc_bytes(Q.n_q, db.sp.s) > scratch_len) return cudaErrorInvalidValue;
    const ClassifyScratch sc = classify_scratch_carve(scratch, Q.n_q, db.sp.s, NOALLOC_LARGE_WARPS);
    return classify_enqueue(db, Q, t, sc, s, nullptr);
}

cudaError_t classify_autotune(const ClassifyDb& db, const ClassifyQuery& Q, const ClassifyScratch& sc, uint32_t reps,
                              cudaStream_t s, Tuning* best, std::vector<TuneRecord>* records) {
    cudaError_t e = cudaSuccess;
    if (Q.n_q == 0 || Q.n_q > sc.chunk || reps == 0) return cudaErrorInvalidValue;
    cudaEvent_t a = nullptr, b = nullptr;
    if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&b)) != cudaSuccess) {
        cudaEventDestroy(a);
        return e;
    }
    uint32_t* qc = queue_counters(sc);
    Tuning cur = DEFAULT_TUNING;
    float best_ms = 0;
    auto timed = [&](auto&& body, float* ms) -> cudaError_t {
        cudaError_t err;
        float total = 0;
        for (uint32_t r = 0; r <= reps; ++r) {  // run 0 warms up
            if ((err = cudaEventRecord(a, s)) != cudaSuccess) return err;
            if ((err = body()) != cudaSuccess) return err;
            if ((err = cudaEventRecord(b, s)) != cudaSuccess) return err;
            if ((err = cudaEventSynchronize(b)) != cudaSuccess) return err;
            float x = 0;
            if ((err = cudaEventElapsedTime(&x, a, b)) != cudaSuccess) return err;
            if (r) total += x;
        }
        *ms = total / reps;
        return cudaSuccess;
    };
    // stage 0: lookup settings
    {
        bool first = true;
        Tuning bl = cur;
        for (uint32_t lb : {2u, 4u, 8u}) {
            for (uint32_t lw : {4u, 8u}) {
                Tuning t = cur;
                t.probe_batch = lb;
                t.lookup_warps = lw;
                Geometry g;
                if ((e = geometry(db, t, sc, &g)) != cudaSuccess) goto done;
                float ms = 0;
                e = timed(
                    [&]() -> cudaError_t {
                        cudaError_t err = cudaMemsetAsync(qc, 0, 2 * sizeof(uint32_t), s);
                        return err != cudaSuccess ? err : launch_lookup(g, db, Q, sc, 0, s);
                    },
                    &ms);
                if (e != cudaSuccess) goto done;
                if (records) records->push_back(TuneRecord{t, 0, ms});
                if (first || ms < best_ms) {
                    best_ms = ms;
                    bl = t;
                    first = false;
                }
            }
        }
        cur = bl;
    }
    // lookup output of the chosen setting, and its queue length, for stage 1
    {
        Geometry g;
        if ((e = geometry(db, cur, sc, &g)) != cudaSuccess) goto done;
        if ((e = cudaMemsetAsync(qc, 0, 2 * sizeof(uint32_t), s)) != cudaSuccess) goto done;
        if ((e = launch_lookup(g, db, Q, sc, 0, s)) != cudaSuccess) goto done;
        if ((e = cudaMemcpyAsync(qc + 4, qc, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)) != cudaSuccess) goto done;
    }
    // stage 1: score settings (with the large path they leave)
    {
        bool first = true;
        Tuning bs = cur;
        for (uint32_t ka : {256u, 512u, 1024u}) {
            for (uint32_t gb : {4u, 8u, 16u}) {
                for (uint32_t sw : {2u, 4u}) {
                    Tuning t = cur;
                    t.score_mode = SCORE_HASH;
                    t.hist_slots = ka;
                    t.gather_batch = gb;
                    t.score_warps = sw;
                    Geometry g;
                    if ((e = geometry(db, t, sc, &g)) != cudaSuccess) goto done;
                    float ms = 0;
                    e = timed(
                        [&]() -> cudaError_t {
                            cudaError_t err;
                            if ((err = cudaMemcpyAsync(qc, qc + 4, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)) !=
                                cudaSuccess)
                                return err;
                            if ((err = cudaMemsetAsync(qc + 1, 0, sizeof(uint32_t), s)) != cudaSuccess) return err;
                            if ((err = launch_score(g, db, Q, sc, 0, s)) != cudaSuccess) return err;
                            return launch_large(g, db, Q, sc, s);
                        },
                        &ms);
                    if (e != cudaSuccess) goto done;
                    if (records) records->push_back(TuneRecord{t, 1, ms});
                    if (first || ms < best_ms) {
                        best_ms = ms;
                        bs = t;
                        first = false;
                    }
                }
            }
        }
        // the sort path, for each largest size class
        if (db.jbits) {
            for (uint32_t smax : {256u, 512u, 1024u, 2048u}) {
                Tuning t = cur;
                t.score_mode = SCORE_SORT;
                t.sort_max = smax;
                t.wide_keys = 0;
                Geometry g;
                if ((e = geometry(db, t, sc, &g)) != cudaSuccess) goto done;
                float ms = 0;
                e = timed(
                    [&]() -> cudaError_t {
                        cudaError_t err;
                        if ((err = cudaMemcpyAsync(qc, qc + 4, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)) !=
                            cudaSuccess)
                            return err;
                        if ((err = cudaMemsetAsync(qc + 1, 0, sizeof(uint32_t), s)) != cudaSuccess) return err;
                        if ((err = launch_score(g, db, Q, sc, 0, s)) != cudaSuccess) return err;
                        return launch_large(g, db, Q, sc, s);
                    },
                    &ms);
                if (e != cudaSuccess) goto done;
                if (records) records->push_back(TuneRecord{t, 1, ms});
                if (ms < best_ms) {
                    best_ms = ms;
                    bs = t;
                }
            }
        }
        cur = bs;
    }
    *best = cur;
done:
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return e;
}

}  // namespace mc
