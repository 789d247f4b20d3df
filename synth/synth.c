/*
 * Seeded synthetic inputs: genomes, taxonomies and reads shaped like the
 * workloads of the MetaCache-GPU evaluation (Section 6, Tables 1 and 2).
 *
 * This module holds none of the classification method's arithmetic: it only
 * draws random bases, substitutions, indels and read placements.  It is
 * shared by the CPU oracle tests and the CUDA path as an input generator.
 *
 * Random numbers: xoshiro256** (Blackman and Vigna, public domain
 * definition), seeded per sub-stream through splitmix64.  Every genome and
 * every read has its own sub-stream, so the output does not depend on the
 * number of threads.  Only integer arithmetic and IEEE basic operations are
 * used (no libm), and the file is compiled with -ffp-contract=off, so x86_64
 * and aarch64 builds produce identical bytes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64(uint64_t* x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void rng_init(rng_t* r, uint64_t seed, uint64_t stream) {
    uint64_t x = seed * 0x9E3779B97F4A7C15ull ^ (stream + 1) * 0xD1B54A32D192ED03ull;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t* r) {
    uint64_t* s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
    s[2] ^= t; s[3] = rotl(s[3], 45);
    return result;
}

/* uniform double in [0,1) with 53 random bits */
static inline double rng_unif(rng_t* r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* uniform integer in [0,n) (multiply-shift, bias < n / 2^64) */
static inline uint64_t rng_below(rng_t* r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

/* approximately standard normal: Irwin-Hall sum of 12 uniforms minus 6 */
static double rng_normal(rng_t* r) {
    double acc = 0.0;
    for (int i = 0; i < 12; ++i) acc += rng_unif(r);
    return acc - 6.0;
}

/* exp(x) from basic IEEE operations only: x = n*ln2 + y, |y| <= ln2/2,
 * exp(y) by its Taylor series (terms < 2^-60 are dropped). */
static double det_exp(double x) {
    const double ln2 = 0.69314718055994530942;
    double nf = x / ln2;
    long n = (long)(nf < 0 ? nf - 0.5 : nf + 0.5);
    double y = x - (double)n * ln2;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 24; ++i) { term = term * y / (double)i; sum += term; }
    while (n > 0) { sum *= 2.0; --n; }
    while (n < 0) { sum *= 0.5; ++n; }
    return sum;
}

static const char BASES[4] = {'A', 'C', 'G', 'T'};

static inline char complement_ascii(char c) {
    switch (c) {
        case 'A': return 'T'; case 'C': return 'G';
        case 'G': return 'C'; case 'T': return 'A';
        case 'a': return 't'; case 'c': return 'g';
        case 'g': return 'c'; case 't': return 'a';
        default: return 'N';
    }
}

/* base with P(G)=P(C)=gc/2, P(A)=P(T)=(1-gc)/2 */
static inline char draw_base(rng_t* r, double gc) {
    double u = rng_unif(r);
    if (u < gc) return (u < 0.5 * gc) ? 'G' : 'C';
    return (u < gc + 0.5 * (1.0 - gc)) ? 'A' : 'T';
}

/* a uniformly chosen base different from c */
static inline char other_base(rng_t* r, char c) {
    int idx = 0;
    for (int i = 0; i < 4; ++i) if (BASES[i] == c) idx = i;
    int k = (int)rng_below(r, 3);
    return BASES[(idx + 1 + k) & 3];
}

/* ------------------------------------------------------------ threading */
typedef void (*item_fn)(void* ctx, uint64_t item);
typedef struct {
    item_fn fn; void* ctx; uint64_t n; uint64_t next; uint64_t chunk; pthread_mutex_t mu;
} pool_t;

static void* pool_worker(void* arg) {
    pool_t* p = (pool_t*)arg;
    for (;;) {
        pthread_mutex_lock(&p->mu);
        uint64_t i = p->next;
        if (i < p->n) p->next = i + p->chunk;
        pthread_mutex_unlock(&p->mu);
        if (i >= p->n) break;
        uint64_t end = i + p->chunk < p->n ? i + p->chunk : p->n;
        for (; i < end; ++i) p->fn(p->ctx, i);
    }
    return NULL;
}

static void par_for(uint64_t n, item_fn fn, void* ctx, int n_threads) {
    if (n_threads <= 1 || n <= 1) {
        for (uint64_t i = 0; i < n; ++i) fn(ctx, i);
        return;
    }
    if (n_threads > 256) n_threads = 256;
    pool_t p; p.fn = fn; p.ctx = ctx; p.n = n; p.next = 0;
    p.chunk = n / ((uint64_t)n_threads * 16);
    if (p.chunk < 1) p.chunk = 1;
    pthread_mutex_init(&p.mu, NULL);
    pthread_t th[256];
    int started = 0;
    for (int t = 0; t < n_threads; ++t)
        if (pthread_create(&th[t], NULL, pool_worker, &p) == 0) ++started;
    if (started == 0) pool_worker(&p);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&p.mu);
}

/* ------------------------------------------------------------- genomes */

/* n i.i.d. bases with GC fraction gc, sub-stream (seed, stream). */
void synth_fill_iid(uint64_t seed, uint64_t stream, uint64_t n, double gc, char* out) {
    rng_t r; rng_init(&r, seed, stream);
    for (uint64_t i = 0; i < n; ++i) out[i] = draw_base(&r, gc);
}

/* copy with each base substituted with probability d by a uniformly chosen
 * different base */
void synth_mutate(uint64_t seed, uint64_t stream, const char* in, uint64_t n, double d, char* out) {
    rng_t r; rng_init(&r, seed, stream);
    for (uint64_t i = 0; i < n; ++i) {
        char c = in[i];
        out[i] = (rng_unif(&r) < d) ? other_base(&r, c) : c;
    }
}

/* Per-genus parameters: length ~ round(exp(N(mu, sigma))) clamped to
 * [min_len, max_len], GC ~ U(gc_lo, gc_hi). */
void synth_genus_params(uint64_t seed, uint64_t n_genera, double mu, double sigma,
                        uint64_t min_len, uint64_t max_len, double gc_lo, double gc_hi,
                        uint64_t* out_len, double* out_gc) {
    for (uint64_t g = 0; g < n_genera; ++g) {
        rng_t r; rng_init(&r, seed, 0x1000000000ull + g);
        double z = rng_normal(&r);
        double l = det_exp(mu + sigma * z);
        uint64_t L = (uint64_t)(l + 0.5);
        if (L < min_len) L = min_len;
        if (L > max_len) L = max_len;
        out_len[g] = L;
        out_gc[g] = gc_lo + (gc_hi - gc_lo) * rng_unif(&r);
    }
}

typedef struct {
    uint64_t seed;
    const uint64_t* len;        /* per genus */
    const double* gc;           /* per genus */
    uint32_t species;           /* species per genus */
    uint32_t strains;           /* strains per species */
    double d_lo, d_hi;          /* species divergence from the genus root */
    double d_strain;            /* extra substitutions per strain */
    char* blob;
    const uint64_t* genus_off;  /* first byte of each genus block in blob */
    /* held-out species copies (generated but never inserted) */
    const uint32_t* held_genus; /* genus index per held-out genome, or NULL */
    uint32_t n_held;
    char* held_blob;
    const uint64_t* held_off;
} genera_ctx;

static void genus_item(void* vctx, uint64_t g) {
    genera_ctx* c = (genera_ctx*)vctx;
    uint64_t L = c->len[g];
    char* root = (char*)malloc(L ? L : 1);
    char* sp = (char*)malloc(L ? L : 1);
    synth_fill_iid(c->seed, 0x2000000000ull + g, L, c->gc[g], root);
    char* dst = c->blob + c->genus_off[g];
    for (uint32_t s = 0; s < c->species; ++s) {
        uint64_t sid = g * c->species + s;
        rng_t r; rng_init(&r, c->seed, 0x3000000000ull + sid);
        double d = c->d_lo + (c->d_hi - c->d_lo) * rng_unif(&r);
        synth_mutate(c->seed, 0x4000000000ull + sid, root, L, d, sp);
        for (uint32_t t = 0; t < c->strains; ++t) {
            uint64_t tid = sid * c->strains + t;
            synth_mutate(c->seed, 0x5000000000ull + tid, sp, L, c->d_strain, dst);
            dst += L;
        }
    }
    for (uint32_t h = 0; h < c->n_held; ++h) {
        if (c->held_genus[h] != g) continue;
        rng_t r; rng_init(&r, c->seed, 0x6000000000ull + h);
        double d = c->d_lo + (c->d_hi - c->d_lo) * rng_unif(&r);
        synth_mutate(c->seed, 0x7000000000ull + h, root, L, d, c->held_blob + c->held_off[h]);
    }
    free(root); free(sp);
}

/* All strains of all genera, genus-major, species-major within a genus.
 * genus_off[g] = byte offset of genus g's first strain (caller-computed:
 * sum over previous genera of species*strains*len).  Held-out genomes are
 * further species copies of their genus root. */
void synth_fill_genera(uint64_t seed, uint64_t n_genera, const uint64_t* len, const double* gc,
                       uint32_t species, uint32_t strains, double d_lo, double d_hi, double d_strain,
                       char* blob, const uint64_t* genus_off,
                       uint32_t n_held, const uint32_t* held_genus, char* held_blob,
                       const uint64_t* held_off, int n_threads) {
    genera_ctx c;
    c.seed = seed; c.len = len; c.gc = gc; c.species = species; c.strains = strains;
    c.d_lo = d_lo; c.d_hi = d_hi; c.d_strain = d_strain; c.blob = blob; c.genus_off = genus_off;
    c.held_genus = held_genus; c.n_held = n_held; c.held_blob = held_blob; c.held_off = held_off;
    par_for(n_genera, genus_item, &c, n_threads);
}

typedef struct {
    uint64_t seed; uint64_t stream_base; const uint64_t* len; const double* gc;
    char* blob; const uint64_t* off;
} iid_ctx;

static void iid_item(void* vctx, uint64_t i) {
    iid_ctx* c = (iid_ctx*)vctx;
    synth_fill_iid(c->seed, c->stream_base + i, c->len[i], c->gc[i], c->blob + c->off[i]);
}

/* n independent sequences, sequence i of length len[i] at blob+off[i]. */
void synth_fill_iid_many(uint64_t seed, uint64_t stream_base, uint64_t n, const uint64_t* len,
                         const double* gc, char* blob, const uint64_t* off, int n_threads) {
    iid_ctx c; c.seed = seed; c.stream_base = stream_base; c.len = len; c.gc = gc;
    c.blob = blob; c.off = off;
    par_for(n, iid_item, &c, n_threads);
}

/* Repeat-rich (eukaryote-like) genomes: built from segments of `seg` bases;
 * segment k is, with probability p_rep, a copy of a uniformly chosen
 * earlier segment of the same genome with substitutions at rate d_rep;
 * else, with probability p_sat, a satellite array (tandem copies of the
 * genome's own i.i.d. unit of sat_period bases, each copy with
 * substitutions at rate d_sat); else i.i.d. bases with the genome's GC.
 * Copies keep their own offset, so a repeat starts at a different phase of
 * the window grid whenever seg is not a multiple of the window stride. */
typedef struct {
    uint64_t seed; uint64_t stream_base; const uint64_t* len; const double* gc;
    uint64_t seg; double p_rep, d_rep;
    double p_sat; uint64_t sat_period; double d_sat;
    char* blob; const uint64_t* off;
} rep_ctx;

static void rep_item(void* vctx, uint64_t i) {
    rep_ctx* c = (rep_ctx*)vctx;
    rng_t r; rng_init(&r, c->seed, c->stream_base + i);
    char* g = c->blob + c->off[i];
    const uint64_t L = c->len[i];
    char unit[1024];
    const uint64_t per = c->sat_period < sizeof unit ? c->sat_period : sizeof unit;
    for (uint64_t x = 0; x < per; ++x) unit[x] = draw_base(&r, c->gc[i]);
    for (uint64_t k = 0, pos = 0; pos < L; ++k, pos += c->seg) {
        const uint64_t n = (L - pos < c->seg) ? L - pos : c->seg;
        const double u = rng_unif(&r);
        if (k > 0 && u < c->p_rep) {
            const uint64_t src = rng_below(&r, k) * c->seg;
            for (uint64_t x = 0; x < n; ++x) {
                char b = g[src + x];
                g[pos + x] = (rng_unif(&r) < c->d_rep) ? other_base(&r, b) : b;
            }
        } else if (per && u < c->p_rep + c->p_sat) {
            for (uint64_t x = 0; x < n; ++x) {
                char b = unit[x % per];
                g[pos + x] = (rng_unif(&r) < c->d_sat) ? other_base(&r, b) : b;
            }
        } else {
            for (uint64_t x = 0; x < n; ++x) g[pos + x] = draw_base(&r, c->gc[i]);
        }
    }
}

void synth_fill_repeat_rich(uint64_t seed, uint64_t stream_base, uint64_t n, const uint64_t* len,
                            const double* gc, uint64_t seg, double p_rep, double d_rep, double p_sat,
                            uint64_t sat_period, double d_sat, char* blob, const uint64_t* off, int n_threads) {
    rep_ctx c; c.seed = seed; c.stream_base = stream_base; c.len = len; c.gc = gc; c.seg = seg;
    c.p_rep = p_rep; c.d_rep = d_rep; c.p_sat = p_sat; c.sat_period = sat_period; c.d_sat = d_sat;
    c.blob = blob; c.off = off;
    par_for(n, rep_item, &c, n_threads);
}

/* --------------------------------------------------------------- reads */
typedef struct {
    uint64_t seed;
    const char* blob; const uint64_t* goff; uint32_t n_main;   /* inserted genomes */
    const char* hblob; const uint64_t* hoff; uint32_t n_held;  /* held-out genomes */
    double held_frac;
    int paired;
    uint32_t len_lo, len_hi;        /* read (mate) length, uniform */
    double frag_a, frag_b;          /* fragment mean = frag_a*len + frag_b */
    double frag_sd_rel, frag_sd_abs;/* fragment sd = frag_sd_rel*mean + frag_sd_abs */
    double sub, indel;
    uint32_t* qlen;                 /* phase 1 output: mate length per query */
    uint64_t* out_off;              /* per sequence */
    char* out_seq;
    uint32_t* out_truth;
    uint64_t stream_base;
} reads_ctx;

static void read_len_item(void* vctx, uint64_t q) {
    reads_ctx* c = (reads_ctx*)vctx;
    rng_t r; rng_init(&r, c->seed, c->stream_base + 2 * q);
    c->qlen[q] = c->len_lo + (uint32_t)rng_below(&r, (uint64_t)(c->len_hi - c->len_lo) + 1);
}

/* Emit n bases of a simulated read from source stream src (forward over
 * g[pos..] if dir>0, reverse complement over g[..pos] if dir<0), applying
 * substitutions and indels.  If the source runs out, the read is padded
 * with random bases. */
static void emit_read(rng_t* r, const char* g, uint64_t glen, int64_t pos, int dir, uint32_t n,
                      double sub, double indel, char* out) {
    uint32_t o = 0;
    int64_t p = pos;
    while (o < n) {
        int in_range = (p >= 0 && (uint64_t)p < glen);
        if (!in_range) { out[o++] = BASES[rng_below(r, 4)]; continue; }
        char b = g[p];
        if (dir < 0) b = complement_ascii(b);
        double u = rng_unif(r);
        if (u < 0.5 * indel) {              /* insertion of a random base */
            out[o++] = BASES[rng_below(r, 4)];
            continue;
        }
        if (u < indel) { p += dir; continue; } /* deletion of the source base */
        if (rng_unif(r) < sub) b = other_base(r, b);
        out[o++] = b;
        p += dir;
    }
}

static void read_fill_item(void* vctx, uint64_t q) {
    reads_ctx* c = (reads_ctx*)vctx;
    rng_t r; rng_init(&r, c->seed, c->stream_base + 2 * q + 1);
    uint32_t len = c->qlen[q];
    int held = (c->n_held > 0) && (rng_unif(&r) < c->held_frac);
    const char* g; uint64_t glen; uint32_t gid;
    if (held) {
        uint32_t h = (uint32_t)rng_below(&r, c->n_held);
        g = c->hblob + c->hoff[h]; glen = c->hoff[h + 1] - c->hoff[h]; gid = 0xFFFFFFFFu;
    } else {
        gid = (uint32_t)rng_below(&r, c->n_main);
        g = c->blob + c->goff[gid]; glen = c->goff[gid + 1] - c->goff[gid];
    }
    c->out_truth[q] = gid;
    uint64_t seq0 = c->paired ? 2 * q : q;
    char* o1 = c->out_seq + c->out_off[seq0];
    if (!c->paired) {
        uint64_t span = glen > len ? glen - len : 0;
        int64_t start = (int64_t)rng_below(&r, span + 1);
        int rev = (int)(rng_next(&r) & 1);
        if (!rev) emit_read(&r, g, glen, start, +1, len, c->sub, c->indel, o1);
        else emit_read(&r, g, glen, start + (int64_t)len - 1, -1, len, c->sub, c->indel, o1);
        return;
    }
    double mean = c->frag_a * len + c->frag_b;
    double sd = c->frag_sd_rel * mean + c->frag_sd_abs;
    double f = mean + sd * rng_normal(&r);
    int64_t flen = (int64_t)(f + 0.5);
    if (flen < (int64_t)len) flen = len;
    if ((uint64_t)flen > glen) flen = (int64_t)glen;
    uint64_t span = glen - (uint64_t)flen;
    int64_t start = (int64_t)rng_below(&r, span + 1);
    int rev = (int)(rng_next(&r) & 1);
    char* o2 = c->out_seq + c->out_off[seq0 + 1];
    /* mate 1 reads the fragment's first strand from its start, mate 2 the
     * opposite strand from the fragment's end */
    if (!rev) {
        emit_read(&r, g, glen, start, +1, len, c->sub, c->indel, o1);
        emit_read(&r, g, glen, start + flen - 1, -1, len, c->sub, c->indel, o2);
    } else {
        emit_read(&r, g, glen, start + flen - 1, -1, len, c->sub, c->indel, o1);
        emit_read(&r, g, glen, start, +1, len, c->sub, c->indel, o2);
    }
}

/* Reads (single-end) or read pairs.  Two phases in one call: mate lengths
 * are drawn per query, sequence offsets are laid out, then bases are
 * filled.  out_off has n_seq+1 entries (n_seq = n_q or 2*n_q), out_qoff
 * n_q+1 entries.  out_seq must hold n_seq * len_hi bytes.  Returns the
 * number of bases written. */
uint64_t synth_reads(uint64_t seed, uint64_t stream_base, uint64_t n_q,
                     const char* blob, const uint64_t* goff, uint32_t n_main,
                     const char* hblob, const uint64_t* hoff, uint32_t n_held, double held_frac,
                     int paired, uint32_t len_lo, uint32_t len_hi,
                     double frag_a, double frag_b, double frag_sd_rel, double frag_sd_abs,
                     double sub, double indel,
                     char* out_seq, uint64_t* out_off, uint32_t* out_qoff, uint32_t* out_truth,
                     int n_threads) {
    reads_ctx c;
    memset(&c, 0, sizeof c);
    c.seed = seed; c.stream_base = stream_base;
    c.blob = blob; c.goff = goff; c.n_main = n_main;
    c.hblob = hblob; c.hoff = hoff; c.n_held = n_held; c.held_frac = held_frac;
    c.paired = paired; c.len_lo = len_lo; c.len_hi = len_hi;
    c.frag_a = frag_a; c.frag_b = frag_b; c.frag_sd_rel = frag_sd_rel; c.frag_sd_abs = frag_sd_abs;
    c.sub = sub; c.indel = indel;
    c.qlen = (uint32_t*)malloc(sizeof(uint32_t) * (n_q ? n_q : 1));
    c.out_off = out_off; c.out_seq = out_seq; c.out_truth = out_truth;
    par_for(n_q, read_len_item, &c, n_threads);
    uint64_t per = paired ? 2 : 1;
    uint64_t acc = 0;
    out_off[0] = 0;
    for (uint64_t q = 0; q < n_q; ++q) {
        out_qoff[q] = (uint32_t)(q * per);
        for (uint64_t m = 0; m < per; ++m) {
            acc += c.qlen[q];
            out_off[q * per + m + 1] = acc;
        }
    }
    out_qoff[n_q] = (uint32_t)(n_q * per);
    par_for(n_q, read_fill_item, &c, n_threads);
    free(c.qlen);
    return acc;
}
