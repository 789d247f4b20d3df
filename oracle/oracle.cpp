// CPU oracle for the MetaCache-GPU hot path (arXiv 2106.08150).
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
// statement of what the database build and the read classification compute.
// Only the test suite, the smoke check and the benchmark's CPU-baseline leg
// may load it.  The product library (the CUDA path) shares no code, header,
// table or constant with it.
//
// Every function follows the paper's text step by step, in the paper's
// order.  Where the paper is silent, the reading taken is stated beside the
// code (h1, the sliding-window size, tie orders, the label thresholds).
//
// Parity pins (tests/test_oracle_pins.py): the Section 2 worked minhash
// example, brute force over tiny windows, reverse-complement invariance of
// canonical k-mers, exhaustive bijectivity of h1, window tiling, the bucket
// cap on an injected repeat, exhaustive lookup on tiny tables, hand-worked
// LCA cases and classification properties of error-free reads.

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

const uint32_t NO_TAXON = 0xFFFFFFFFu;

struct Params {
    uint32_t k;       // k-mer length (Section 5.2: default 16)
    uint32_t s;       // sketch size (Section 5.2: default 16)
    uint32_t w;       // window length (Section 4.1: windows of size w)
    uint32_t stride;  // window stride (Section 4.1: overlap k-1, stride w-k+1)
    uint32_t cap;     // locations kept per feature (Section 4.1: 254 by default)
};

// Section 5.2 step 1 / Section 5.3: the regular bases A, C, G, T get a
// 2-bit code; everything else (N and other ambiguity letters) is invalid.
// Lower case is treated like upper case.
int base_code(uint8_t c) {
    switch (c) {
        case 'A': case 'a': return 0;
        case 'C': case 'c': return 1;
        case 'G': case 'g': return 2;
        case 'T': case 't': return 3;
        default: return -1;
    }
}

// h1 (Section 4.1: "a hash function h1 is applied" to each canonical k-mer;
// the paper does not name it).  Reading: the "lowbias32" 32-bit integer
// mixer from C. Wellons' hash-prospector (public domain): two rounds of
// xor-shift and odd multiply, a bijection on 32-bit words.
uint32_t h1(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

// Section 4.1: a sequence is divided into windows of w bases that overlap by
// k-1 bases, i.e. window j starts at j*stride.  Window j's k-mers start at
// positions j*stride .. min(j*stride + w - k, L - k).  A window exists while
// its first k-mer fits, so there are ceil((L-k+1)/stride) windows (none if
// L < k).  Window ids are positional: a window without a valid k-mer still
// takes its id.
uint64_t num_windows(uint64_t L, const Params& p) {
    if (L < p.k) return 0;
    return (L - p.k + 1 + p.stride - 1) / p.stride;
}

// Forward code of the k-mer at x[pos..pos+k): the first base is the most
// significant 2-bit digit.  Reverse complement: the bases in reverse order,
// each complemented (code c -> 3-c).  Returns false if any base is invalid.
bool kmer_codes(const uint8_t* x, uint64_t pos, uint32_t k, uint32_t* fwd, uint32_t* rc) {
    uint64_t f = 0, r = 0;
    for (uint32_t i = 0; i < k; ++i) {
        int c = base_code(x[pos + i]);
        if (c < 0) return false;
        f = f * 4 + (uint64_t)c;
    }
    for (uint32_t i = 0; i < k; ++i) {
        int c = base_code(x[pos + k - 1 - i]);
        r = r * 4 + (uint64_t)(3 - c);
    }
    *fwd = (uint32_t)f;
    *rc = (uint32_t)r;
    return true;
}

// Section 4.1 (canonical k-mers): the smaller of a k-mer's code and its
// reverse complement's code, so that a read and its reverse complement
// produce the same k-mers.
uint32_t canonical(uint32_t fwd, uint32_t rc) { return fwd < rc ? fwd : rc; }

// Section 2 and Section 4.1: the minhash sketch of a window is the s smallest
// distinct hash values of its valid canonical k-mers (repeated k-mers count
// once, as in the Section 2 example where ACTG occurs twice).
std::vector<uint32_t> sketch_window(const uint8_t* x, uint64_t L, uint64_t j, const Params& p) {
    std::vector<uint32_t> hashes;
    uint64_t first = j * p.stride;
    uint64_t last = std::min<uint64_t>(first + p.w - p.k, L - p.k);
    for (uint64_t pos = first; pos <= last; ++pos) {
        uint32_t f, r;
        if (!kmer_codes(x, pos, p.k, &f, &r)) continue;  // Section 5.2 step 2: valid k-mers only
        hashes.push_back(h1(canonical(f, r)));
    }
    std::sort(hashes.begin(), hashes.end());
    hashes.erase(std::unique(hashes.begin(), hashes.end()), hashes.end());
    if (hashes.size() > p.s) hashes.resize(p.s);
    return hashes;
}

// A location is (target id, window id), packed so that numeric order is
// (target, window) order.
uint64_t make_loc(uint32_t t, uint32_t j) { return ((uint64_t)t << 32) | j; }

struct DB {
    Params p;
    uint32_t n_targets = 0;
    uint64_t n_windows = 0;
    uint64_t n_pairs = 0;       // (feature, location) pairs offered to the table
    uint64_t overflow_keys = 0; // features that had more than cap locations
    // Section 4.1: each feature maps to a bucket of locations, limited to cap.
    std::unordered_map<uint32_t, std::vector<uint64_t>> buckets;
    // locations of each feature before the cap (for the shards after this one)
    std::unordered_map<uint32_t, uint64_t> uncapped;
};

struct TargetSketches {
    std::vector<std::vector<uint32_t>> win;  // sketch per window
};

}  // namespace

extern "C" {

uint32_t oracle_h1(uint32_t x) { return h1(x); }

uint64_t oracle_num_windows(uint64_t L, uint32_t k, uint32_t stride) {
    Params p{k, 1, k, stride, 1};
    return num_windows(L, p);
}

// Codes of one k-mer (for pin tests).  Returns 0 if it has an invalid base.
int oracle_kmer(const char* x, uint32_t k, uint32_t* fwd, uint32_t* rc, uint32_t* canon) {
    uint32_t f, r;
    if (!kmer_codes((const uint8_t*)x, 0, k, &f, &r)) return 0;
    *fwd = f; *rc = r; *canon = canonical(f, r);
    return 1;
}

// Test mode for the Section 2 worked example: the k-mers of a window taken
// forward (canonical = 0) or canonical (canonical = 1), hashed through a
// caller table lut[code] (4^k entries) instead of h1, then the s smallest
// distinct values.  Returns the sketch size.
uint32_t oracle_sketch_custom(const char* window, uint32_t len, uint32_t k, uint32_t s, int use_canonical,
                              const uint32_t* lut, uint32_t* out) {
    std::vector<uint32_t> hashes;
    for (uint64_t pos = 0; pos + k <= len; ++pos) {
        uint32_t f, r;
        if (!kmer_codes((const uint8_t*)window, pos, k, &f, &r)) continue;
        uint32_t key = use_canonical ? canonical(f, r) : f;
        hashes.push_back(lut ? lut[key] : h1(key));
    }
    std::sort(hashes.begin(), hashes.end());
    hashes.erase(std::unique(hashes.begin(), hashes.end()), hashes.end());
    if (hashes.size() > s) hashes.resize(s);
    for (size_t i = 0; i < hashes.size(); ++i) out[i] = hashes[i];
    return (uint32_t)hashes.size();
}

// Sketches of every window of every sequence.  win_offs[i] = first window
// of sequence i (n_seq+1 entries).  sketch[w*s + i], cnt[w].  Returns the
// total number of windows; with null outputs it only counts.
uint64_t oracle_sketch(uint32_t k, uint32_t s, uint32_t w, uint32_t stride, uint64_t n_seq, const char* seq,
                       const uint64_t* offs, uint64_t* win_offs, uint32_t* sketch, uint32_t* cnt) {
    Params p{k, s, w, stride, 1};
    uint64_t total = 0;
    for (uint64_t i = 0; i < n_seq; ++i) {
        uint64_t L = offs[i + 1] - offs[i];
        uint64_t nw = num_windows(L, p);
        if (win_offs) win_offs[i] = total;
        if (sketch && cnt) {
            for (uint64_t j = 0; j < nw; ++j) {
                std::vector<uint32_t> f = sketch_window((const uint8_t*)seq + offs[i], L, j, p);
                cnt[total + j] = (uint32_t)f.size();
                for (uint32_t q = 0; q < s; ++q) sketch[(total + j) * s + q] = q < f.size() ? f[q] : 0;
            }
        }
        total += nw;
    }
    if (win_offs) win_offs[n_seq] = total;
    return total;
}

// Database build (Section 4.1 build phase, Section 5.2 build pipeline):
// targets get ids in input order; for every target t, every window j and
// every feature f of window j's sketch, the location (t, j) is added to f's
// bucket.  Finally each bucket is sorted and cut to the cap, keeping the
// smallest locations (the CPU version's behaviour, since it inserts in
// ascending (target, window) order, Section 4.1).
// key_filter (sorted, optional) restricts the stored features to a subset,
// which lets tests check sampled keys of a large database.
// Sketching may use n_threads threads (per-target work); the insertion is
// one thread in target order.
//
// Partitioned databases (Section 4.3: the targets are split over GPUs, each
// building a database of its own targets): target_base is the global id of
// this shard's first target, so its locations carry global ids.  The
// shards hold contiguous id ranges in order, so the cap smallest locations
// of a feature over all targets are the earlier shards' first; with the
// earlier shards' location counts prior(f) (prior_keys ascending), this
// shard keeps at most max(0, cap - prior(f)) of its own, and the shards
// together hold exactly the database of all targets.  (Reading: the paper
// caps each partition on its own; the single-database cap is kept here so
// that sharded results equal the unsharded ones.)  overflow_keys counts
// the features whose locations here and in the prior exceed cap.
void* oracle_db_build_shard(uint32_t k, uint32_t s, uint32_t w, uint32_t stride, uint32_t cap, uint32_t n_targets,
                            const char* seq, const uint64_t* offs, const uint32_t* key_filter, uint64_t n_filter,
                            int n_threads, uint32_t target_base, const uint32_t* prior_keys,
                            const uint32_t* prior_counts, uint64_t n_prior) {
    DB* db = new DB;
    db->p = Params{k, s, w, stride, cap};
    db->n_targets = n_targets;
    std::vector<TargetSketches> sk(n_targets);
    auto work = [&](uint32_t t) {
        uint64_t L = offs[t + 1] - offs[t];
        uint64_t nw = num_windows(L, db->p);
        sk[t].win.resize(nw);
        for (uint64_t j = 0; j < nw; ++j)
            sk[t].win[j] = sketch_window((const uint8_t*)seq + offs[t], L, j, db->p);
    };
    if (n_threads <= 1) {
        for (uint32_t t = 0; t < n_targets; ++t) work(t);
    } else {
        std::vector<std::thread> pool;
        std::atomic_uint next{0};
        for (int i = 0; i < n_threads; ++i)
            pool.emplace_back([&] {
                for (;;) {
                    uint32_t t = next.fetch_add(1);
                    if (t >= n_targets) break;
                    work(t);
                }
            });
        for (auto& th : pool) th.join();
    }
    for (uint32_t t = 0; t < n_targets; ++t) {
        for (uint64_t j = 0; j < sk[t].win.size(); ++j) {
            db->n_windows++;
            for (uint32_t f : sk[t].win[j]) {
                db->n_pairs++;
                if (key_filter && !std::binary_search(key_filter, key_filter + n_filter, f)) continue;
                db->buckets[f].push_back(make_loc(target_base + t, (uint32_t)j));
            }
        }
        sk[t].win.clear();
        sk[t].win.shrink_to_fit();
    }
    for (auto it = db->buckets.begin(); it != db->buckets.end();) {
        std::vector<uint64_t>& b = it->second;
        std::sort(b.begin(), b.end());
        db->uncapped[it->first] = b.size();
        uint64_t prior = 0;
        if (n_prior) {
            const uint32_t* p = std::lower_bound(prior_keys, prior_keys + n_prior, it->first);
            if (p != prior_keys + n_prior && *p == it->first) prior = prior_counts[p - prior_keys];
        }
        const uint64_t limit = prior >= cap ? 0 : cap - prior;
        if (prior + b.size() > cap) db->overflow_keys++;
        if (b.size() > limit) b.resize(limit);
        if (b.empty()) it = db->buckets.erase(it);
        else ++it;
    }
    return db;
}

void* oracle_db_build(uint32_t k, uint32_t s, uint32_t w, uint32_t stride, uint32_t cap, uint32_t n_targets,
                      const char* seq, const uint64_t* offs, const uint32_t* key_filter, uint64_t n_filter,
                      int n_threads) {
    return oracle_db_build_shard(k, s, w, stride, cap, n_targets, seq, offs, key_filter, n_filter, n_threads, 0,
                                 nullptr, nullptr, 0);
}

// Features of a database and their location counts before the cap, clamped
// to cap (what a later shard needs), ascending.  Returns the number of
// features; with null outputs it only counts.
uint64_t oracle_db_feature_counts(void* h, uint32_t* keys, uint32_t* counts) {
    DB* db = (DB*)h;
    std::vector<uint32_t> ks;
    for (auto& kv : db->uncapped) ks.push_back(kv.first);
    std::sort(ks.begin(), ks.end());
    for (size_t i = 0; i < ks.size() && keys; ++i) {
        keys[i] = ks[i];
        counts[i] = (uint32_t)std::min<uint64_t>(db->uncapped[ks[i]], db->p.cap);
    }
    return ks.size();
}

void oracle_db_free(void* h) { delete (DB*)h; }

// out: n_targets, n_windows, n_pairs, n_keys, n_locations, overflow_keys
void oracle_db_stats(void* h, uint64_t* out) {
    DB* db = (DB*)h;
    uint64_t locs = 0;
    for (auto& kv : db->buckets) locs += kv.second.size();
    out[0] = db->n_targets;
    out[1] = db->n_windows;
    out[2] = db->n_pairs;
    out[3] = db->buckets.size();
    out[4] = locs;
    out[5] = db->overflow_keys;
}

// Bucket of one feature: number of locations (written to out up to max).
uint64_t oracle_db_lookup(void* h, uint32_t key, uint64_t* out, uint64_t max) {
    DB* db = (DB*)h;
    auto it = db->buckets.find(key);
    if (it == db->buckets.end()) return 0;
    for (uint64_t i = 0; i < it->second.size() && i < max; ++i) out[i] = it->second[i];
    return it->second.size();
}

// Features in [lo, hi) in ascending order with their buckets.  keys/counts
// get one entry per feature, locs the concatenated buckets.  With null
// buffers only the sizes are returned (*n_locs_out).  Returns #features.
uint64_t oracle_db_dump(void* h, uint64_t lo, uint64_t hi, uint32_t* keys, uint32_t* counts, uint64_t* locs,
                        uint64_t* n_locs_out) {
    DB* db = (DB*)h;
    std::vector<uint32_t> ks;
    for (auto& kv : db->buckets)
        if (kv.first >= lo && kv.first < hi) ks.push_back(kv.first);
    std::sort(ks.begin(), ks.end());
    uint64_t nl = 0;
    for (size_t i = 0; i < ks.size(); ++i) {
        const std::vector<uint64_t>& b = db->buckets[ks[i]];
        if (keys) keys[i] = ks[i];
        if (counts) counts[i] = (uint32_t)b.size();
        if (locs) for (uint64_t v : b) locs[nl++] = v; else nl += b.size();
    }
    if (n_locs_out) *n_locs_out = nl;
    return ks.size();
}

// Lowest common ancestor (Section 4.2: candidates close to the maximum are
// labelled with the LCA of their taxa).  Plain walk: compute both depths by
// following parents to the root (parent == self), lift the deeper node to
// the same depth, then lift both until they meet.  Different roots, an
// out-of-range id or NO_TAXON give NO_TAXON.
uint32_t oracle_lca(uint32_t n_taxa, const uint32_t* parent, uint32_t a, uint32_t b) {
    if (a >= n_taxa || b >= n_taxa) return NO_TAXON;
    auto depth = [&](uint32_t x) {
        uint32_t d = 0;
        while (parent[x] != x && d <= n_taxa) { x = parent[x]; ++d; }
        return d;
    };
    uint32_t da = depth(a), db = depth(b);
    while (da > db) { a = parent[a]; --da; }
    while (db > da) { b = parent[b]; --db; }
    while (a != b) {
        if (parent[a] == a) return NO_TAXON;  // both are (different) roots
        a = parent[a];
        b = parent[b];
    }
    return a;
}

struct Cand { uint32_t score, t, j0, j1; };

// Sliding-window size (Section 5.6: "determined by the length of the
// respective read"; the formula is not given).  Reading: the number of
// consecutive windows that the k-mer starts of a fragment spanning `span`
// bases can touch, span = read length (single-end) or max(sum of mate
// lengths, max_insert) (pairs): ceil((span-k)/stride) + 1, 0 if span < k.
uint64_t oracle_sws(uint32_t n_mates, uint64_t span_sum, uint32_t max_insert, uint32_t k, uint32_t stride) {
    uint64_t span = n_mates <= 1 ? span_sum : std::max<uint64_t>(span_sum, max_insert);
    return span >= k ? (span - k + stride - 1) / stride + 1 : 0;
}

// Step 6 of classification (Section 4.2 and Section 6.5 hit threshold), on
// the top-m candidates in order (score descending, target ascending): no
// candidate or top score < hits_min -> unclassified; else the candidates
// within lca_band_pct percent of the top score are "close": one -> its
// target's taxon, several -> the LCA of their taxa.  hits = top score (0
// without candidates), top_target = top target (NO_TAXON without).
void assign_label(const std::vector<Cand>& cands, uint32_t n_taxa, const uint32_t* parent,
                  const uint32_t* taxon_of_target, uint32_t hits_min, uint32_t lca_band_pct, uint32_t* label,
                  uint32_t* hits, uint32_t* top_target) {
    if (cands.empty()) {
        *label = NO_TAXON;
        *hits = 0;
        if (top_target) *top_target = NO_TAXON;
        return;
    }
    const Cand& top = cands[0];
    *hits = top.score;
    if (top_target) *top_target = top.t;
    if (top.score < hits_min) {
        *label = NO_TAXON;
        return;
    }
    std::vector<uint32_t> close;
    for (const Cand& c : cands)
        if (100ull * c.score >= (uint64_t)(100 - lca_band_pct) * top.score) close.push_back(c.t);
    uint32_t lab = taxon_of_target[close[0]];
    for (size_t i = 1; i < close.size(); ++i) lab = oracle_lca(n_taxa, parent, lab, taxon_of_target[close[i]]);
    *label = lab;
}

// Merge of partitioned results (Section 4.2: with a partitioned database
// the top candidates of every partition are merged).  lists[l] holds, per
// query, m candidates {score, global target, j0, j1} (score 0 = unused) of
// partition l.  A target lives in one partition, so the global top m are
// the m best of the union (score descending, target ascending), labelled
// by the same rule as oracle_classify.  cands_out (optional) as there.
void oracle_merge(uint32_t n_lists, const uint32_t* const* lists, uint32_t m, uint32_t n_q, uint32_t n_taxa,
                  const uint32_t* parent, const uint32_t* taxon_of_target, uint32_t hits_min, uint32_t lca_band_pct,
                  uint32_t* label, uint32_t* hits, uint32_t* top_target, uint32_t* cands_out) {
    for (uint32_t q = 0; q < n_q; ++q) {
        std::vector<Cand> all;
        for (uint32_t l = 0; l < n_lists; ++l)
            for (uint32_t i = 0; i < m; ++i) {
                const uint32_t* c = lists[l] + ((uint64_t)q * m + i) * 4;
                if (c[0]) all.push_back(Cand{c[0], c[1], c[2], c[3]});
            }
        std::sort(all.begin(), all.end(), [](const Cand& a, const Cand& b) {
            if (a.score != b.score) return a.score > b.score;
            return a.t < b.t;
        });
        if (all.size() > m) all.resize(m);
        if (cands_out)
            for (uint32_t i = 0; i < m; ++i) {
                uint32_t* o = cands_out + ((uint64_t)q * m + i) * 4;
                if (i < all.size()) { o[0] = all[i].score; o[1] = all[i].t; o[2] = all[i].j0; o[3] = all[i].j1; }
                else { o[0] = 0; o[1] = NO_TAXON; o[2] = 0; o[3] = 0; }
            }
        assign_label(all, n_taxa, parent, taxon_of_target, hits_min, lca_band_pct, &label[q], &hits[q],
                     top_target ? &top_target[q] : nullptr);
    }
}

// Read classification (Section 4.2 query phase; Section 5.2 query steps 1-8).
// Per query (one read or one read pair = consecutive mates qoffs[q] ..
// qoffs[q+1]):
//  1. every mate is cut into windows exactly like a target (Section 4.2:
//     "windows of the same length as used in the database") and each
//     window is sketched;
//  2. every feature of every window is looked up and its bucket appended
//     (reading: windows are looked up independently, so a feature in two
//     windows of one query contributes its bucket twice);
//  3. the location list is sorted and identical locations are accumulated
//     into the window count statistic (location -> hit count);
//  4. sliding window (Section 4.2, Section 5.6): for every location (t, j0)
//     of the statistic, score = sum of counts of (t, j) with
//     j0 <= j <= j0 + sws - 1.  Reading for sws (the paper says only that it
//     follows from the read length): span = read length (single-end) or
//     max(sum of mate lengths, max_insert) (pairs); sws = ceil((span-k)/stride)
//     + 1, the most windows a fragment of that span can touch;
//  5. top m (Section 4.2): one candidate per target (its best range; ties ->
//     smaller j0), ordered by score descending then target ascending;
//  6. label (Section 4.2 and Section 6.5 hit threshold): no candidate or
//     top score < hits_min -> unclassified.  Otherwise the candidates whose
//     score is within lca_band_pct percent of the top score are "close"; one
//     close candidate -> its target's taxon ("difference above a
//     threshold"), several -> the LCA of their taxa.
// Outputs: label, hits (top score, 0 without candidates), top_target
// (NO_TAXON without candidates).  stats (optional, 3 per query): features
// looked up, locations gathered, distinct locations.  cands_out (optional,
// m x {score, target, j0, j1} per query; unused slots score 0, target
// NO_TAXON), j1 = the last window present in the candidate's range.
void oracle_classify(void* h, uint32_t n_taxa, const uint32_t* parent, const uint32_t* taxon_of_target,
                     uint32_t m, uint32_t hits_min, uint32_t lca_band_pct, uint32_t max_insert,
                     const char* seq, const uint64_t* offs, uint32_t n_q, const uint32_t* qoffs,
                     uint32_t* label, uint32_t* hits, uint32_t* top_target, uint64_t* stats, uint32_t* cands_out,
                     int n_threads) {
    DB* db = (DB*)h;
    const Params& p = db->p;
    auto one = [&](uint32_t q) {
        std::vector<uint64_t> found;
        uint64_t n_features = 0;
        uint64_t span_sum = 0;
        uint32_t n_mates = qoffs[q + 1] - qoffs[q];
        for (uint32_t i = qoffs[q]; i < qoffs[q + 1]; ++i) {
            uint64_t L = offs[i + 1] - offs[i];
            span_sum += L;
            uint64_t nw = num_windows(L, p);
            for (uint64_t j = 0; j < nw; ++j) {
                std::vector<uint32_t> f = sketch_window((const uint8_t*)seq + offs[i], L, j, p);
                for (uint32_t x : f) {
                    ++n_features;
                    auto it = db->buckets.find(x);
                    if (it != db->buckets.end()) found.insert(found.end(), it->second.begin(), it->second.end());
                }
            }
        }
        std::sort(found.begin(), found.end());
        std::vector<std::pair<uint64_t, uint32_t>> stat;  // window count statistic
        for (uint64_t v : found) {
            if (!stat.empty() && stat.back().first == v) stat.back().second++;
            else stat.push_back({v, 1});
        }
        uint64_t sws = oracle_sws(n_mates, span_sum, max_insert, p.k, p.stride);
        std::map<uint32_t, Cand> best;  // per target
        for (size_t i = 0; i < stat.size(); ++i) {
            uint32_t t = (uint32_t)(stat[i].first >> 32);
            uint64_t j0 = stat[i].first & 0xFFFFFFFFu;
            Cand c{0, t, (uint32_t)j0, (uint32_t)j0};
            for (size_t l = i; l < stat.size(); ++l) {
                uint32_t tl = (uint32_t)(stat[l].first >> 32);
                uint64_t jl = stat[l].first & 0xFFFFFFFFu;
                if (tl != t || jl >= j0 + sws) break;
                c.score += stat[l].second;
                c.j1 = (uint32_t)jl;
            }
            auto it = best.find(t);
            if (it == best.end() || c.score > it->second.score ||
                (c.score == it->second.score && c.j0 < it->second.j0))
                best[t] = c;
        }
        std::vector<Cand> cands;
        for (auto& kv : best) cands.push_back(kv.second);
        std::sort(cands.begin(), cands.end(), [](const Cand& a, const Cand& b) {
            if (a.score != b.score) return a.score > b.score;
            return a.t < b.t;
        });
        if (cands.size() > m) cands.resize(m);
        if (cands_out) {
            for (uint32_t i = 0; i < m; ++i) {
                uint32_t* o = cands_out + ((uint64_t)q * m + i) * 4;
                if (i < cands.size()) { o[0] = cands[i].score; o[1] = cands[i].t; o[2] = cands[i].j0; o[3] = cands[i].j1; }
                else { o[0] = 0; o[1] = NO_TAXON; o[2] = 0; o[3] = 0; }
            }
        }
        if (stats) {
            stats[3 * (uint64_t)q + 0] = n_features;
            stats[3 * (uint64_t)q + 1] = found.size();
            stats[3 * (uint64_t)q + 2] = stat.size();
        }
        assign_label(cands, n_taxa, parent, taxon_of_target, hits_min, lca_band_pct, &label[q], &hits[q],
                     top_target ? &top_target[q] : nullptr);
    };
    if (n_threads <= 1) {
        for (uint32_t q = 0; q < n_q; ++q) one(q);
    } else {
        std::vector<std::thread> pool;
        std::atomic_uint next{0};
        const uint32_t chunk = 64;
        for (int i = 0; i < n_threads; ++i)
            pool.emplace_back([&] {
                for (;;) {
                    uint32_t b = next.fetch_add(chunk);
                    if (b >= n_q) break;
                    uint32_t e = std::min<uint32_t>(n_q, b + chunk);
                    for (uint32_t q = b; q < e; ++q) one(q);
                }
            });
        for (auto& th : pool) th.join();
    }
}

}  // extern "C"
