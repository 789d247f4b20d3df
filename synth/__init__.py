"""Seeded synthetic workloads shaped like the MetaCache-GPU evaluation inputs.

The paper evaluates on RefSeq 202 / AFS31 reference sets (Table 1) and the
HiSeq, MiSeq and KAL_D read sets (Table 2).  None of those are available
here, so this module builds stand-ins with the same structure: genomes of a
few Mbp organised in genera of related strains, a taxonomy over them, and
single-end or paired-end short reads with sequencing errors.

It is the one module shared by the CPU oracle tests and the CUDA path, and
it holds none of the classification method's arithmetic (no encoding,
k-mers, hashing, sketching or scoring): only random bases, substitutions,
indels and read placement, drawn by `synth.c`.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None

NO_GENOME = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so next to it (plain C, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, u32, dbl, i32, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                  ctypes.c_int, ctypes.c_void_p)
        lib.synth_fill_iid.argtypes = [u64, u64, u64, dbl, vp]
        lib.synth_genus_params.argtypes = [u64, u64, dbl, dbl, u64, u64, dbl, dbl, vp, vp]
        lib.synth_fill_genera.argtypes = [u64, u64, vp, vp, u32, u32, dbl, dbl, dbl, vp, vp,
                                          u32, vp, vp, vp, i32]
        lib.synth_fill_iid_many.argtypes = [u64, u64, u64, vp, vp, vp, vp, i32]
        lib.synth_fill_repeat_rich.argtypes = [u64, u64, u64, vp, vp, u64, dbl, dbl, dbl, u64, dbl, vp, vp, i32]
        lib.synth_reads.argtypes = [u64, u64, u64, vp, vp, u32, vp, vp, u32, dbl, i32, u32, u32,
                                    dbl, dbl, dbl, dbl, dbl, dbl, vp, vp, vp, vp, i32]
        lib.synth_reads.restype = u64
        _lib = lib
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data


def _threads() -> int:
    return max(1, os.cpu_count() or 1)


@dataclass
class Workload:
    """One synthetic build+classify workload (host arrays)."""
    name: str
    genomes: np.ndarray          # uint8 ASCII, all targets concatenated
    goffs: np.ndarray            # uint64 [n_targets+1]
    parent: np.ndarray           # uint32 [n_taxa], root has parent == itself
    taxon_of_target: np.ndarray  # uint32 [n_targets]
    reads: np.ndarray            # uint8 ASCII, all mates concatenated
    roffs: np.ndarray            # uint64 [n_seq+1]
    qoffs: np.ndarray            # uint32 [n_queries+1]; query q = mates qoffs[q]..qoffs[q+1]
    truth: np.ndarray            # uint32 [n_queries] source target or NO_GENOME
    db_params: dict = field(default_factory=dict)
    cls_params: dict = field(default_factory=dict)
    recipe: str = ""
    # genomes generated but not inserted (new species of existing genera):
    # (ASCII blob, offsets, taxon of each); their species taxa are in parent
    held: tuple | None = None

    @property
    def n_targets(self) -> int:
        return len(self.goffs) - 1

    @property
    def n_bp(self) -> int:
        return int(self.goffs[-1])

    @property
    def n_queries(self) -> int:
        return len(self.qoffs) - 1

    @property
    def n_seq(self) -> int:
        return len(self.roffs) - 1


DB_PARAMS = dict(k=16, sketch_size=16, window_len=128, window_stride=113, bucket_cap=254)
CLS_PARAMS = dict(max_candidates=4, hits_min=4, lca_band_pct=10, max_insert=0)


def iid_genomes(seed: int, lengths, gc=0.5, stream_base: int = 0x8000000000) -> tuple[np.ndarray, np.ndarray]:
    """Independent i.i.d. genomes with the given lengths."""
    lib = _load()
    lens = np.ascontiguousarray(lengths, dtype=np.uint64)
    gcs = np.full(len(lens), gc, dtype=np.float64) if np.isscalar(gc) else np.ascontiguousarray(gc, np.float64)
    offs = np.zeros(len(lens) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    blob = np.empty(int(offs[-1]), dtype=np.uint8)
    starts = np.ascontiguousarray(offs[:-1])
    lib.synth_fill_iid_many(seed, stream_base, len(lens), _p(lens), _p(gcs), _p(blob), _p(starts), _threads())
    return blob, offs


def simulate_reads(seed: int, n_q: int, genomes: np.ndarray, goffs: np.ndarray, *, paired: bool,
                   len_lo: int, len_hi: int, sub: float, indel: float = 0.0,
                   frag_a: float = 0.0, frag_b: float = 0.0, frag_sd_rel: float = 0.0,
                   frag_sd_abs: float = 0.0, held: tuple | None = None, held_frac: float = 0.0,
                   stream_base: int = 0x9000000000):
    """Reads sampled from `genomes` (uniform genome, uniform start, random
    strand).  Paired: fragment ~ N(frag_a*len+frag_b, frag_sd_rel*mean+frag_sd_abs)
    clamped to [len, genome length]; mate 1 from the fragment's start, mate 2
    the reverse complement of its end."""
    lib = _load()
    per = 2 if paired else 1
    n_seq = n_q * per
    seq = np.empty(max(1, n_seq * len_hi), dtype=np.uint8)
    roffs = np.zeros(n_seq + 1, dtype=np.uint64)
    qoffs = np.zeros(n_q + 1, dtype=np.uint32)
    truth = np.zeros(max(1, n_q), dtype=np.uint32)
    hblob, hoffs = (None, None) if held is None else held
    n_held = 0 if held is None else len(hoffs) - 1
    total = lib.synth_reads(seed, stream_base, n_q, _p(genomes), _p(goffs), len(goffs) - 1,
                            _p(hblob), _p(hoffs), n_held, held_frac, int(paired), len_lo, len_hi,
                            frag_a, frag_b, frag_sd_rel, frag_sd_abs, sub, indel,
                            _p(seq), _p(roffs), _p(qoffs), _p(truth), _threads())
    return seq[:total].copy(), roffs, qoffs, truth[:n_q].copy()


def _concat_reads(parts):
    seqs, roffs_l, qoffs_l, truth_l = [], [], [], []
    base_b, base_s = 0, 0
    for seq, roffs, qoffs, truth in parts:
        seqs.append(seq)
        roffs_l.append(roffs[:-1] + np.uint64(base_b))
        qoffs_l.append(qoffs[:-1] + np.uint32(base_s))
        truth_l.append(truth)
        base_b += int(roffs[-1])
        base_s += len(roffs) - 1
    return (np.concatenate(seqs), np.append(np.concatenate(roffs_l), np.uint64(base_b)).astype(np.uint64),
            np.append(np.concatenate(qoffs_l), np.uint32(base_s)).astype(np.uint32), np.concatenate(truth_l))


def tiny_workload(seed: int = 1000, n_reads: int = 10_000, n_decoys: int = 1_000) -> Workload:
    """Tiny build+classify: 8 i.i.d. genomes of 200 kbp, taxonomy root -> 2
    genera -> 2 species each -> 2 strains each (targets are strains), 10k
    single-end 100 bp reads with 1% substitutions plus 1k i.i.d. decoys."""
    genomes, goffs = iid_genomes(seed, [200_000] * 8)
    # taxa: 0 root; 1,2 genera; 3..6 species; 7..14 strains
    parent = np.array([0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 5, 5, 6, 6], dtype=np.uint32)
    taxon = np.arange(7, 15, dtype=np.uint32)
    r = simulate_reads(seed, n_reads, genomes, goffs, paired=False, len_lo=100, len_hi=100, sub=0.01)
    dblob, doffs = iid_genomes(seed + 7, [100] * n_decoys, stream_base=0xA000000000)
    d = (dblob, doffs, np.arange(n_decoys + 1, dtype=np.uint32), np.full(n_decoys, NO_GENOME, np.uint32))
    reads, roffs, qoffs, truth = _concat_reads([r, d])
    return Workload("tiny-8x200kbp-11kSE100", genomes, goffs, parent, taxon, reads, roffs, qoffs, truth,
                    dict(DB_PARAMS), dict(CLS_PARAMS, max_insert=0),
                    recipe="8 iid uniform-ACGT genomes x 200 kbp; 3-level taxonomy; 10k SE 100 bp reads, "
                           "uniform start, random strand, 1% substitutions; 1k iid 100 bp decoys")


def genera_workload(seed: int, *, n_families: int, genera_per_family: int, species: int, strains: int,
                    median_len: float, sigma: float, min_len: int, max_len: int,
                    gc_lo: float = 0.3, gc_hi: float = 0.7, d_lo: float = 0.01, d_hi: float = 0.05,
                    d_strain: float = 0.001, held_genera: int = 0, held_per_genus: int = 0):
    """Genera of related genomes: each genus has an i.i.d. root with its own
    GC; each species is a mutated copy of the root; each strain a further
    0.1%-mutated copy of its species.  Taxonomy root -> families -> genera ->
    species -> strains; targets are the strains.  Returns (genomes, goffs,
    parent, taxon_of_target, held) with held = (blob, offs, taxon) of the
    held-out species copies (each a species taxon of its genus that has no
    inserted target), or None."""
    lib = _load()
    n_genera = n_families * genera_per_family
    lens = np.zeros(n_genera, dtype=np.uint64)
    gcs = np.zeros(n_genera, dtype=np.float64)
    lib.synth_genus_params(seed, n_genera, math.log(median_len), sigma, min_len, max_len, gc_lo, gc_hi,
                           _p(lens), _p(gcs))
    per_genus = species * strains
    genus_off = np.zeros(n_genera, dtype=np.uint64)
    genus_off[1:] = np.cumsum(lens * np.uint64(per_genus))[:-1]
    total = int((lens * np.uint64(per_genus)).sum())
    blob = np.empty(total, dtype=np.uint8)
    tlens = np.repeat(lens, per_genus)
    goffs = np.zeros(len(tlens) + 1, dtype=np.uint64)
    goffs[1:] = np.cumsum(tlens)
    # held-out: further species copies of evenly spaced genera, never inserted
    held_genus = np.array([g for g in np.linspace(0, n_genera - 1, held_genera, dtype=np.int64)
                           for _ in range(held_per_genus)], dtype=np.uint32) if held_genera else np.zeros(0, np.uint32)
    hlens = lens[held_genus] if len(held_genus) else np.zeros(0, np.uint64)
    hoffs = np.zeros(len(hlens) + 1, dtype=np.uint64)
    hoffs[1:] = np.cumsum(hlens)
    hblob = np.empty(max(1, int(hoffs[-1])), dtype=np.uint8)
    hstarts = np.ascontiguousarray(hoffs[:-1])
    lib.synth_fill_genera(seed, n_genera, _p(lens), _p(gcs), species, strains, d_lo, d_hi, d_strain,
                          _p(blob), _p(genus_off), len(held_genus), _p(held_genus), _p(hblob),
                          _p(hstarts), _threads())
    # taxonomy ids: 0 root | families | genera | species | strains
    fam0 = 1
    gen0 = fam0 + n_families
    sp0 = gen0 + n_genera
    st0 = sp0 + n_genera * species
    n_taxa = st0 + n_genera * species * strains
    parent = np.zeros(n_taxa, dtype=np.uint32)
    parent[fam0:gen0] = 0
    g = np.arange(n_genera)
    parent[gen0 + g] = fam0 + g // genera_per_family
    s = np.arange(n_genera * species)
    parent[sp0 + s] = gen0 + s // species
    t = np.arange(n_genera * species * strains)
    parent[st0 + t] = sp0 + t // strains
    taxon = (st0 + t).astype(np.uint32)
    held = None
    if len(held_genus):
        held_taxon = np.arange(n_taxa, n_taxa + len(held_genus), dtype=np.uint32)
        parent = np.concatenate([parent, (gen0 + held_genus).astype(np.uint32)])
        held = (hblob[:int(hoffs[-1])], hoffs, held_taxon)
    return blob, goffs, parent, taxon, held


def mid_workload(seed: int = 1001, *, n_pairs: int = 10_000_000, n_families: int = 10, genera_per_family: int = 10,
            len_scale: float = 1.0, held_genera: int = 5, held_per_genus: int = 10) -> Workload:
    """Mid-size build+classify: 1,000 genomes (100 genera x 5 species x 2
    strains), genus length lognormal (median 3 Mbp, sigma 0.5), GC U(0.3,0.7),
    species at 1-5% substitution divergence from the genus root, 4-level
    taxonomy; 10M paired-end 2x150 bp reads, fragment N(300, 30), 0.5%
    substitutions and 0.05% indels, 5% from held-out genomes.
    `len_scale`, `n_families`, `n_pairs` shrink it for tests."""
    median = 3e6 * len_scale
    blob, goffs, parent, taxon, held = genera_workload(
        seed, n_families=n_families, genera_per_family=genera_per_family, species=5, strains=2,
        median_len=median, sigma=0.5, min_len=max(1000, int(20_000 * len_scale)),
        max_len=int(60e6 * len_scale), held_genera=held_genera, held_per_genus=held_per_genus)
    reads, roffs, qoffs, truth = simulate_reads(
        seed, n_pairs, blob, goffs, paired=True, len_lo=150, len_hi=150, sub=0.005, indel=0.0005,
        frag_b=300.0, frag_sd_abs=30.0, held=None if held is None else held[:2],
        held_frac=0.05 if held is not None else 0.0)
    name = "mid-1000genomes-10Mpairs" if (len_scale == 1.0 and n_families == 10 and n_pairs == 10_000_000) \
        else f"scaled-{n_families * genera_per_family * 10}genomes-x{len_scale:g}-{n_pairs}pairs"
    return Workload(name, blob, goffs, parent, taxon, reads, roffs, qoffs, truth,
                    dict(DB_PARAMS), dict(CLS_PARAMS, max_insert=390),
                    recipe="genera of related genomes (lognormal length, GC U(0.3,0.7), species 1-5% "
                           "divergent, strains +0.1%); 2x150 bp pairs, fragment N(300,30), 0.5% sub, "
                           "0.05% indel, 5% from held-out species", held=held)


def mixed_batches(seed: int, genomes: np.ndarray, goffs: np.ndarray, *, n_batches: int = 256,
                  median: float = 5e4, sigma: float = 1.0, lo: int = 1000, hi: int = 2_000_000,
                  len_lo: int = 50, len_hi: int = 300, sub: float = 0.005, indel: float = 0.0005,
                  sizes=None, held: tuple | None = None, held_frac: float = 0.0):
    """Query batches of uneven size and read length: batch sizes lognormal
    (median, sigma) clamped to [lo, hi] (or the given `sizes`); in each batch
    half the queries are single-end reads and half are pairs, read length
    uniform in [len_lo, len_hi] (both mates of a pair alike), fragment
    N(1.5 * len + 50, 0.1 * mean).  Returns a list of (reads, roffs, qoffs,
    truth) per batch, each with its own offsets."""
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = np.clip(np.round(np.exp(rng.normal(math.log(median), sigma, n_batches))), lo, hi).astype(np.int64)
    out = []
    for b, n in enumerate(sizes):
        n = int(n)
        n_se = n // 2
        parts = []
        if n_se:
            parts.append(simulate_reads(seed * 7919 + 2 * b, n_se, genomes, goffs, paired=False, len_lo=len_lo,
                                        len_hi=len_hi, sub=sub, indel=indel, stream_base=0xA000000000,
                                        held=None if held is None else held[:2], held_frac=held_frac))
        if n - n_se:
            parts.append(simulate_reads(seed * 7919 + 2 * b + 1, n - n_se, genomes, goffs, paired=True,
                                        len_lo=len_lo, len_hi=len_hi, sub=sub, indel=indel, frag_a=1.5,
                                        frag_b=50.0, frag_sd_rel=0.1, stream_base=0xB000000000,
                                        held=None if held is None else held[:2], held_frac=held_frac))
        if not parts:
            out.append((np.zeros(0, np.uint8), np.zeros(1, np.uint64), np.zeros(1, np.uint32),
                        np.zeros(0, np.uint32)))
        else:
            out.append(_concat_reads(parts))
    return out


def concat_batches(batches):
    """One (reads, roffs, qoffs, truth) holding all batches in order."""
    return _concat_reads(batches)


def repeat_rich_genomes(seed: int, lengths, gcs, seg: int = 5000, p_rep: float = 0.3, d_rep: float = 0.005,
                        p_sat: float = 0.02, sat_period: int = 171, d_sat: float = 0.02,
                        stream_base: int = 0xC000000000) -> tuple[np.ndarray, np.ndarray]:
    """Eukaryote-like genomes of the given lengths: 5 kbp segments, each with
    probability p_rep a copy (d_rep substitutions) of an earlier segment of
    the same genome placed at its own offset, with probability p_sat a
    satellite array (tandem copies of the genome's own sat_period-base unit,
    d_sat substitutions per copy), else i.i.d. with the genome's GC.
    Returns (blob, offsets)."""
    lib = _load()
    lens = np.ascontiguousarray(lengths, dtype=np.uint64)
    gc = np.ascontiguousarray(gcs, dtype=np.float64)
    offs = np.zeros(len(lens) + 1, dtype=np.uint64)
    offs[1:] = np.cumsum(lens)
    blob = np.empty(max(1, int(offs[-1])), dtype=np.uint8)
    starts = np.ascontiguousarray(offs[:-1])
    lib.synth_fill_repeat_rich(seed, stream_base, len(lens), _p(lens), _p(gc), seg, p_rep, d_rep, p_sat,
                               sat_period, d_sat, _p(blob), _p(starts), _threads())
    return blob[:int(offs[-1])], offs


def large_workload(seed: int = 1002, *, scaled: bool = True, n_pairs: int = 50_000_000, n_families: int = 98,
                   genera_per_family: int = 10, n_euk: int = 200, len_scale: float = 1.0,
                   euk_scale: float = 1.0, held_genera: int = 0, held_per_genus: int = 10) -> Workload:
    """Large single-GPU database: genera of bacterial-like genomes as in the
    mid workload (980 genera x 5 species x 2 strains = 9,800 genomes) plus
    n_euk repeat-rich eukaryote-like genomes of U(50, 200) Mbp (30% of 5 kbp
    segments repeated with 0.5% substitutions, 2% satellite arrays of a
    171-base unit), which overfill buckets.
    scaled=True shrinks the bacterial median to 1.1 Mbp and the eukaryote
    lengths x0.1 (about 15 Gbp in all instead of about 58).  Taxonomy: the
    mid-workload tree plus one family of eukaryote genera (10 species per
    genus, one target per species).  Reads: pairs as in the mid workload.
    held_genera > 0 also generates held_per_genus not-inserted species
    copies of that many genera (Workload.held), for live extension."""
    median = (1.1e6 if scaled else 3e6) * len_scale
    blob, goffs, parent, taxon, held = genera_workload(
        seed, n_families=n_families, genera_per_family=genera_per_family, species=5, strains=2,
        median_len=median, sigma=0.5, min_len=max(1000, int(20_000 * len_scale)), max_len=int(60e6 * len_scale),
        held_genera=held_genera, held_per_genus=held_per_genus)
    rng = np.random.default_rng(seed)
    f = (0.1 if scaled else 1.0) * euk_scale
    elens = np.round(rng.uniform(50e6, 200e6, n_euk) * f).astype(np.uint64)
    egc = rng.uniform(0.3, 0.7, n_euk)
    eblob, eoffs = repeat_rich_genomes(seed, elens, egc)
    genomes = np.concatenate([blob, eblob])
    del blob
    goffs = np.concatenate([goffs, eoffs[1:] + goffs[-1]]).astype(np.uint64)
    # taxonomy: family -> n_euk / 10 genera -> species (= targets)
    n_taxa = len(parent)
    n_eg = max(1, (n_euk + 9) // 10)
    fam = n_taxa
    gen = np.arange(fam + 1, fam + 1 + n_eg, dtype=np.uint32)
    sp = np.arange(fam + 1 + n_eg, fam + 1 + n_eg + n_euk, dtype=np.uint32)
    parent = np.concatenate([parent, np.array([0], np.uint32), np.full(n_eg, fam, np.uint32),
                             gen[np.arange(n_euk) // 10]]).astype(np.uint32)
    taxon = np.concatenate([taxon, sp]).astype(np.uint32)
    reads, roffs, qoffs, truth = simulate_reads(
        seed, n_pairs, genomes, goffs, paired=True, len_lo=150, len_hi=150, sub=0.005, indel=0.0005,
        frag_b=300.0, frag_sd_abs=30.0)
    n_t = len(goffs) - 1
    name = f"large-{n_t}genomes-{int(goffs[-1]) / 1e9:.1f}Gbp-{n_pairs}pairs" + ("-scaled" if scaled else "")
    return Workload(name, genomes, goffs, parent, taxon, reads, roffs, qoffs, truth,
                    dict(DB_PARAMS), dict(CLS_PARAMS, max_insert=390),
                    recipe="mid-workload genera (980 genera x 10 genomes) + repeat-rich eukaryote-like genomes "
                           "U(50,200) Mbp (30% of 5 kbp segments repeated, 0.5% sub; 2% satellite arrays of a "
                           "171-base unit, 2% sub)"
                           + (", bacterial median 1.1 Mbp and eukaryotes x0.1" if scaled else ""), held=held)
