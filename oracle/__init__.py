"""CPU oracle for the MetaCache-GPU hot path -- TEST INFRASTRUCTURE ONLY.

`oracle.cpp` states, in plain C++17, what database build and read
classification compute (arXiv 2106.08150, Sections 2, 4.1, 4.2 and 5.2-5.6).
Only the tests, `__graft_entry__.smoke()` and the CPU-baseline / reference
legs of `bench.py` may use it.  The CUDA product path never imports it, and
the two share no code.

Parity status: every function is pinned by `tests/test_oracle_pins.py`
(worked example of Section 2, brute force, closed forms and invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
NO_TAXON = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so next to it (plain C++, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        lib.oracle_h1.argtypes, lib.oracle_h1.restype = [u32], u32
        lib.oracle_num_windows.argtypes, lib.oracle_num_windows.restype = [u64, u32, u32], u64
        lib.oracle_kmer.argtypes, lib.oracle_kmer.restype = [ctypes.c_char_p, u32, vp, vp, vp], i32
        lib.oracle_sketch_custom.argtypes = [ctypes.c_char_p, u32, u32, u32, i32, vp, vp]
        lib.oracle_sketch_custom.restype = u32
        lib.oracle_sketch.argtypes = [u32, u32, u32, u32, u64, vp, vp, vp, vp, vp]
        lib.oracle_sketch.restype = u64
        lib.oracle_db_build.argtypes = [u32, u32, u32, u32, u32, u32, vp, vp, vp, u64, i32]
        lib.oracle_db_build.restype = vp
        lib.oracle_db_build_shard.argtypes = [u32, u32, u32, u32, u32, u32, vp, vp, vp, u64, i32, u32, vp, vp, u64]
        lib.oracle_db_build_shard.restype = vp
        lib.oracle_db_feature_counts.argtypes, lib.oracle_db_feature_counts.restype = [vp, vp, vp], u64
        lib.oracle_merge.argtypes = [u32, vp, u32, u32, u32, vp, vp, u32, u32, vp, vp, vp, vp]
        lib.oracle_db_free.argtypes = [vp]
        lib.oracle_db_stats.argtypes = [vp, vp]
        lib.oracle_db_lookup.argtypes, lib.oracle_db_lookup.restype = [vp, u32, vp, u64], u64
        lib.oracle_db_dump.argtypes, lib.oracle_db_dump.restype = [vp, u64, u64, vp, vp, vp, vp], u64
        lib.oracle_lca.argtypes, lib.oracle_lca.restype = [u32, vp, u32, u32], u32
        lib.oracle_sws.argtypes, lib.oracle_sws.restype = [u32, u64, u32, u32, u32], u64
        lib.oracle_classify.argtypes = [vp, u32, vp, vp, u32, u32, u32, u32, vp, vp, u32, vp, vp, vp, vp, vp, vp,
                                        i32]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _u8(x) -> np.ndarray:
    if isinstance(x, (bytes, bytearray)):
        return np.frombuffer(bytes(x), dtype=np.uint8).copy()
    if isinstance(x, str):
        return np.frombuffer(x.encode(), dtype=np.uint8).copy()
    return np.ascontiguousarray(x, dtype=np.uint8)


def h1(x: int) -> int:
    return int(_load().oracle_h1(x))


def num_windows(L: int, k: int, stride: int) -> int:
    return int(_load().oracle_num_windows(L, k, stride))


def kmer(s: str, k: int):
    """(fwd, rc, canonical) codes of the first k-mer of s, or None if invalid."""
    f, r, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    ok = _load().oracle_kmer(s.encode(), k, ctypes.byref(f), ctypes.byref(r), ctypes.byref(c))
    return (f.value, r.value, c.value) if ok else None


def sketch_custom(window: str, k: int, s: int, canonical: bool, lut=None) -> list[int]:
    out = np.zeros(max(1, len(window)), dtype=np.uint32)
    lut_a = None if lut is None else np.ascontiguousarray(lut, dtype=np.uint32)
    n = _load().oracle_sketch_custom(window.encode(), len(window), k, s, int(canonical), _p(lut_a), _p(out))
    return [int(v) for v in out[:n]]


def sketch(seq, offs, *, k, sketch_size, window_len, window_stride, **_):
    """Sketches of every window of every sequence: (win_offs, sketch[n_win, s], cnt[n_win])."""
    lib = _load()
    seq = _u8(seq)
    offs = np.ascontiguousarray(offs, dtype=np.uint64)
    n_seq = len(offs) - 1
    win_offs = np.zeros(n_seq + 1, dtype=np.uint64)
    n = lib.oracle_sketch(k, sketch_size, window_len, window_stride, n_seq, _p(seq), _p(offs), _p(win_offs),
                          None, None)
    sk = np.zeros((max(1, n), sketch_size), dtype=np.uint32)
    cnt = np.zeros(max(1, n), dtype=np.uint32)
    lib.oracle_sketch(k, sketch_size, window_len, window_stride, n_seq, _p(seq), _p(offs), _p(win_offs),
                      _p(sk), _p(cnt))
    return win_offs, sk[:n], cnt[:n]


class DB:
    """Oracle database: feature -> sorted locations (target<<32 | window), capped."""

    def __init__(self, seq, offs, *, k, sketch_size, window_len, window_stride, bucket_cap,
                 key_filter=None, n_threads: int = 1, target_base: int = 0, prior=None, **_):
        """A database of the targets seq/offs.  For one partition (shard) of
        a partitioned database: target_base = the global id of its first
        target, prior = (features ascending, counts) of the earlier shards'
        locations (see oracle_db_build_shard)."""
        lib = _load()
        self._seq = _u8(seq)
        self._offs = np.ascontiguousarray(offs, dtype=np.uint64)
        self.params = dict(k=k, sketch_size=sketch_size, window_len=window_len, window_stride=window_stride,
                           bucket_cap=bucket_cap)
        kf = None if key_filter is None else np.unique(np.ascontiguousarray(key_filter, dtype=np.uint32))
        pk = pc = None
        if prior is not None:
            pk = np.ascontiguousarray(prior[0], dtype=np.uint32)
            pc = np.ascontiguousarray(prior[1], dtype=np.uint32)
        self._h = lib.oracle_db_build_shard(k, sketch_size, window_len, window_stride, bucket_cap,
                                            len(self._offs) - 1, _p(self._seq), _p(self._offs), _p(kf),
                                            0 if kf is None else len(kf), n_threads, target_base, _p(pk), _p(pc),
                                            0 if pk is None else len(pk))
        self._lib = lib

    def feature_counts(self):
        """(features ascending, location counts before the cap clamped to the cap)."""
        n = self._lib.oracle_db_feature_counts(self._h, None, None)
        keys = np.zeros(max(1, n), dtype=np.uint32)
        counts = np.zeros(max(1, n), dtype=np.uint32)
        self._lib.oracle_db_feature_counts(self._h, _p(keys), _p(counts))
        return keys[:n], counts[:n]

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.oracle_db_free(self._h)
            self._h = None

    def stats(self) -> dict:
        out = np.zeros(6, dtype=np.uint64)
        self._lib.oracle_db_stats(self._h, _p(out))
        return dict(zip(["n_targets", "n_windows", "n_pairs", "n_keys", "n_locations", "overflow_keys"],
                        map(int, out)))

    def lookup(self, key: int) -> np.ndarray:
        out = np.zeros(1 << 16, dtype=np.uint64)
        n = self._lib.oracle_db_lookup(self._h, key, _p(out), len(out))
        return out[:n].copy()

    def dump(self, lo: int = 0, hi: int = 1 << 32):
        """(keys, counts, locs) of features in [lo, hi), ascending."""
        nl = ctypes.c_uint64()
        nk = self._lib.oracle_db_dump(self._h, lo, hi, None, None, None, ctypes.byref(nl))
        keys = np.zeros(max(1, nk), dtype=np.uint32)
        counts = np.zeros(max(1, nk), dtype=np.uint32)
        locs = np.zeros(max(1, nl.value), dtype=np.uint64)
        self._lib.oracle_db_dump(self._h, lo, hi, _p(keys), _p(counts), _p(locs), ctypes.byref(nl))
        return keys[:nk], counts[:nk], locs[:nl.value]

    def classify(self, parent, taxon_of_target, reads, roffs, qoffs, *, max_candidates, hits_min, lca_band_pct,
                 max_insert, n_threads: int = 1, with_stats: bool = False, with_cands: bool = False):
        """(label, hits, top_target[, stats[n_q,3]][, cands[n_q,m,4]]) per query."""
        parent = np.ascontiguousarray(parent, dtype=np.uint32)
        tax = np.ascontiguousarray(taxon_of_target, dtype=np.uint32)
        reads = _u8(reads)
        roffs = np.ascontiguousarray(roffs, dtype=np.uint64)
        qoffs = np.ascontiguousarray(qoffs, dtype=np.uint32)
        nq = len(qoffs) - 1
        label = np.zeros(max(1, nq), dtype=np.uint32)
        hits = np.zeros(max(1, nq), dtype=np.uint32)
        top = np.zeros(max(1, nq), dtype=np.uint32)
        stats = np.zeros((max(1, nq), 3), dtype=np.uint64) if with_stats else None
        cands = np.zeros((max(1, nq), max_candidates, 4), dtype=np.uint32) if with_cands else None
        if not 0 <= lca_band_pct <= 100:
            raise ValueError("lca_band_pct must be in 0..100")
        self._lib.oracle_classify(self._h, len(parent), _p(parent), _p(tax), max_candidates, hits_min,
                                  lca_band_pct, max_insert, _p(reads), _p(roffs), nq, _p(qoffs), _p(label),
                                  _p(hits), _p(top), _p(stats), _p(cands), n_threads)
        out = (label[:nq], hits[:nq], top[:nq])
        if with_stats:
            out = out + (stats[:nq],)
        if with_cands:
            out = out + (cands[:nq],)
        return out


def sws(n_mates: int, span_sum: int, max_insert: int, k: int, stride: int) -> int:
    return int(_load().oracle_sws(n_mates, span_sum, max_insert, k, stride))


def lca(parent, a: int, b: int) -> int:
    parent = np.ascontiguousarray(parent, dtype=np.uint32)
    return int(_load().oracle_lca(len(parent), _p(parent), a, b))


def merge(lists, parent, taxon_of_target, *, max_candidates, hits_min, lca_band_pct, **_):
    """Merged classification of a partitioned database: lists = per-shard
    candidate arrays [n_q, m, 4] with global target ids.  Returns (label,
    hits, top_target, cands[n_q, m, 4])."""
    lib = _load()
    arrs = [np.ascontiguousarray(x, dtype=np.uint32) for x in lists]
    nq = arrs[0].shape[0] if arrs else 0
    m = max_candidates
    ptrs = (ctypes.c_void_p * max(1, len(arrs)))(*[a.ctypes.data for a in arrs])
    parent = np.ascontiguousarray(parent, dtype=np.uint32)
    tax = np.ascontiguousarray(taxon_of_target, dtype=np.uint32)
    label = np.zeros(max(1, nq), dtype=np.uint32)
    hits = np.zeros(max(1, nq), dtype=np.uint32)
    top = np.zeros(max(1, nq), dtype=np.uint32)
    cands = np.zeros((max(1, nq), m, 4), dtype=np.uint32)
    lib.oracle_merge(len(arrs), ptrs, m, nq, len(parent), _p(parent), _p(tax), hits_min, lca_band_pct, _p(label),
                     _p(hits), _p(top), _p(cands))
    return label[:nq], hits[:nq], top[:nq], cands[:nq]
