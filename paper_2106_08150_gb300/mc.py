"""Thin Python binding of libmc (include/mc.h): the same entry points, with
arguments marshalled from PyTorch tensors.  Every step of the method runs in
the library's CUDA kernels; PyTorch only provides device memory and streams.

Importing this module fails loudly when libmc.so has not been built: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmc.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "mc.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() (nvcc, sm_103a)")

_lib = ctypes.CDLL(LIB_PATH)

MC_OK, MC_ERR_ARG, MC_ERR_STATE, MC_ERR_OOM, MC_ERR_TABLE_FULL, MC_ERR_TIMEOUT, MC_ERR_CUDA, MC_ERR_CAPACITY = range(8)
MC_NO_TAXON = 0xFFFFFFFF
MC_DEBUG_COUNTERS = 28  # entries of mc_classify_debug's counters
MC_NO_TARGET = 0xFFFFFFFF
MC_MAX_CANDIDATES = 8


class McError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_lib.mc_status_string(code).decode()}: {msg}")
        self.code = code


class mc_db_params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("sketch_size", ctypes.c_uint32), ("window_len", ctypes.c_uint32),
                ("window_stride", ctypes.c_uint32), ("bucket_cap", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("max_locations", ctypes.c_uint64), ("hbm_budget", ctypes.c_uint64)]


class mc_classify_params(ctypes.Structure):
    _fields_ = [("max_candidates", ctypes.c_uint32), ("hits_min", ctypes.c_uint32),
                ("lca_band_pct", ctypes.c_uint32), ("max_insert", ctypes.c_uint32)]


class mc_db_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ["n_targets", "n_windows", "n_pairs", "n_keys", "n_locations", "overflow_keys", "dropped_locations",
                 "table_slots", "max_probe", "device_bytes"]] + \
               [("load_factor", ctypes.c_double), ("finalized", ctypes.c_uint32), ("max_depth", ctypes.c_uint32),
                ("loc_bytes", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class mc_batch(ctypes.Structure):
    _fields_ = [("n_seq", ctypes.c_uint32), ("n_queries", ctypes.c_uint32), ("seq", ctypes.c_void_p),
                ("offs", ctypes.c_void_p), ("qoffs", ctypes.c_void_p), ("label", ctypes.c_void_p),
                ("hits", ctypes.c_void_p), ("top_target", ctypes.c_void_p)]


class mc_tuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in
                ["hist_slots", "probe_batch", "gather_batch", "lookup_warps", "score_warps", "wide_keys", "score_mode",
                 "sort_max"]]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class mc_tuning_time(ctypes.Structure):
    _fields_ = [("tuning", mc_tuning), ("stage", ctypes.c_uint32), ("ms", ctypes.c_float)]


class mc_server_config(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_uint32), ("max_set_queries", ctypes.c_uint32),
                ("max_set_jobs", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("hbm_limit", ctypes.c_uint64)]


class mc_job(ctypes.Structure):
    _fields_ = [("n_seq", ctypes.c_uint32), ("n_queries", ctypes.c_uint32), ("seq", ctypes.c_void_p),
                ("offs", ctypes.c_void_p), ("qoffs", ctypes.c_void_p), ("label", ctypes.c_void_p),
                ("hits", ctypes.c_void_p), ("top_target", ctypes.c_void_p)]


class mc_job_info(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double),
                ("epoch", ctypes.c_uint64), ("pieces", ctypes.c_uint32), ("status", ctypes.c_int)]


class mc_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in
                ["jobs_submitted", "jobs_done", "queries_done", "launch_sets", "extensions", "epoch", "hbm_in_use",
                 "hbm_limit", "hbm_peak"]] + \
               [(n, ctypes.c_double) for n in ["p50_latency_s", "p99_latency_s", "max_latency_s", "busy_s",
                                               "extension_mean_s", "extension_max_s"]]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class mc_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


_vp, _u32, _u64, _i = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_SIGS = {
    "mc_version": ([], _i),
    "mc_last_error_string": ([], ctypes.c_char_p),
    "mc_status_string": ([_i], ctypes.c_char_p),
    "mc_set_allocator": ([ctypes.POINTER(mc_allocator)], _i),
    "mc_db_create": ([ctypes.POINTER(mc_db_params), _u32, _vp, _vp, ctypes.POINTER(_vp)], _i),
    "mc_db_add_targets": ([_vp, _u32, _vp, _vp, _vp, ctypes.POINTER(_u32)], _i),
    "mc_db_finalize": ([_vp], _i),
    "mc_db_feature_counts": ([_vp, _u64, _vp, _vp, ctypes.POINTER(_u64)], _i),
    "mc_db_finalize_after": ([_vp, _u32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_u64)], _i),
    "mc_merge_candidates": ([_vp, ctypes.POINTER(mc_classify_params), _u32, _u32, ctypes.POINTER(_vp),
                             ctypes.POINTER(_u32), _vp, _u32, _vp, _vp, _vp, _vp, _vp], _i),
    "mc_classify": ([_vp, ctypes.POINTER(mc_classify_params), _u32, _vp, _vp, _u32, _vp, _vp, _vp, _vp, _vp], _i),
    "mc_classify_debug": ([_vp, ctypes.POINTER(mc_classify_params), _u32, _vp, _vp, _u32, _vp, _vp, _vp, _vp, _vp,
                           _vp, _vp], _i),
    "mc_classify_status": ([_vp, _vp], _i),
    "mc_classify_noalloc": ([_vp, ctypes.POINTER(mc_classify_params), _u32, _vp, _vp, _u32, _vp, _vp, _vp, _vp,
                             _vp], _i),
    "mc_db_free": ([_vp], None),
    "mc_db_stats": ([_vp, ctypes.POINTER(mc_db_stats_t)], _i),
    "mc_db_dump": ([_vp, _u64, _u64, _u64, _u64, _vp, _vp, _vp, ctypes.POINTER(_u64), ctypes.POINTER(_u64)], _i),
    "mc_window_offsets": ([ctypes.POINTER(mc_db_params), _u32, _vp, _vp, _vp], _i),
    "mc_sketch": ([ctypes.POINTER(mc_db_params), _u32, _vp, _vp, _vp, _u64, _vp, _vp, _vp], _i),
    "mc_db_save": ([_vp, ctypes.c_char_p], _i),
    "mc_db_load": ([ctypes.c_char_p, _vp, ctypes.POINTER(_vp)], _i),
    "mc_db_set_tuning": ([_vp, ctypes.POINTER(mc_tuning)], _i),
    "mc_classify_batches": ([_vp, ctypes.POINTER(mc_classify_params), ctypes.POINTER(mc_tuning), _u32,
                             ctypes.POINTER(mc_batch), _vp], _i),
    "mc_plan_create": ([_vp, ctypes.POINTER(mc_classify_params), ctypes.POINTER(mc_tuning), _u32, _u32,
                        ctypes.POINTER(_vp)], _i),
    "mc_plan_run": ([_vp, _u32, ctypes.POINTER(mc_batch), _vp], _i),
    "mc_plan_kernels": ([_vp], _i),
    "mc_plan_free": ([_vp], None),
    "mc_autotune": ([_vp, ctypes.POINTER(mc_classify_params), _u32, ctypes.POINTER(mc_batch), _u32,
                     ctypes.POINTER(mc_tuning), ctypes.POINTER(mc_tuning_time), _u32, ctypes.POINTER(_u32)], _i),
    "mc_server_create": ([_vp, ctypes.POINTER(mc_classify_params), ctypes.POINTER(mc_server_config),
                          ctypes.POINTER(_vp)], _i),
    "mc_server_submit": ([_vp, ctypes.POINTER(mc_job), ctypes.POINTER(_u64)], _i),
    "mc_server_extend": ([_vp, _u32, _vp, _vp, _vp, ctypes.POINTER(_u32)], _i),
    "mc_server_wait": ([_vp, _u64, ctypes.c_double, ctypes.POINTER(mc_job_info)], _i),
    "mc_server_drain": ([_vp, ctypes.c_double], _i),
    "mc_server_stats_get": ([_vp, ctypes.POINTER(mc_server_stats)], _i),
    "mc_server_free": ([_vp], None),
    "mc_debug_stall_next_sort": ([_u64], _i),
    "mc_trace_enable": ([_i], _i),
    "mc_trace_report": ([ctypes.c_char_p, ctypes.c_size_t, _i], _i),
    "mc_kernel_launches": ([], _u64),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes, _f.restype = _args, _res


def declared_symbols() -> list[str]:
    """Function names declared in include/mc.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|uint64_t|const char\*)\s+(mc_\w+)\s*\(", text, re.M)))


def _check(code: int):
    if code != MC_OK:
        raise McError(code, _lib.mc_last_error_string().decode())


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def db_params(k=16, sketch_size=16, window_len=128, window_stride=113, bucket_cap=254, max_locations=0,
              hbm_budget=0) -> mc_db_params:
    return mc_db_params(k, sketch_size, window_len, window_stride, bucket_cap, 0, max_locations, hbm_budget)


def classify_params(max_candidates=4, hits_min=4, lca_band_pct=10, max_insert=0) -> mc_classify_params:
    return mc_classify_params(max_candidates, hits_min, lca_band_pct, max_insert)


# ------------------------------------------------------------ allocator
_torch_alloc_refs = None


def use_torch_allocator(enable: bool = True):
    """Route every device allocation of the library through PyTorch's
    caching allocator (mc_set_allocator)."""
    global _torch_alloc_refs
    if not enable:
        _check(_lib.mc_set_allocator(None))
        _torch_alloc_refs = None
        return
    import torch

    def _alloc(ctx, size, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None

    def _free(ctx, ptr, size, stream):
        torch.cuda.caching_allocator_delete(ptr)

    a = mc_allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)
    _torch_alloc_refs = a  # keep the callbacks alive
    _check(_lib.mc_set_allocator(ctypes.byref(a)))


# ------------------------------------------------------------- C-ABI calls
def mc_version() -> int:
    return _lib.mc_version()


def mc_db_create(params: mc_db_params, n_taxa: int, parent: np.ndarray, stream=None) -> int:
    parent = np.ascontiguousarray(parent, dtype=np.uint32)
    h = _vp()
    _check(_lib.mc_db_create(ctypes.byref(params), n_taxa, parent.ctypes.data, _stream(stream), ctypes.byref(h)))
    return h.value


def mc_db_add_targets(db: int, n_targets: int, seq, offs, taxon: np.ndarray) -> int:
    taxon = np.ascontiguousarray(taxon, dtype=np.uint32)
    first = _u32()
    _check(_lib.mc_db_add_targets(db, n_targets, _ptr(seq), _ptr(offs), taxon.ctypes.data, ctypes.byref(first)))
    return first.value


def mc_db_finalize(db: int):
    _check(_lib.mc_db_finalize(db))


def mc_db_feature_counts(db: int, keys=None, counts=None, max_keys: int = 0) -> int:
    """Features of the pending targets and their counts (device uint32
    buffers of max_keys entries); returns the number of features (nothing is
    written when they do not fit: call with max_keys = 0 to size them)."""
    n = _u64()
    code = _lib.mc_db_feature_counts(db, max_keys, _ptr(keys), _ptr(counts), ctypes.byref(n))
    if code not in (MC_OK, MC_ERR_CAPACITY) or (code == MC_ERR_CAPACITY and max_keys):
        _check(code)
    return n.value


def mc_db_finalize_after(db: int, prior):
    """prior: [(keys, counts, n)] of the earlier shards (device buffers)."""
    n = len(prior)
    keys = (_vp * max(1, n))(*[_ptr(k) for k, _, _ in prior])
    cnts = (_vp * max(1, n))(*[_ptr(c) for _, c, _ in prior])
    sizes = (_u64 * max(1, n))(*[int(x) for _, _, x in prior])
    _check(_lib.mc_db_finalize_after(db, n, keys, cnts, sizes))


def mc_merge_candidates(db: int, params: mc_classify_params, n_queries: int, cands, target_base, taxon_of_target,
                        n_targets: int, label, hits, top_target=None, cands_out=None, stream=None):
    """cands: device buffers (one per shard) as written by mc_classify_debug."""
    n = len(cands)
    lists = (_vp * max(1, n))(*[_ptr(c) for c in cands])
    base = (_u32 * max(1, n))(*[int(b) for b in target_base])
    _check(_lib.mc_merge_candidates(db, ctypes.byref(params), n_queries, n, lists, base, _ptr(taxon_of_target),
                                    n_targets, _ptr(label), _ptr(hits), _ptr(top_target), _ptr(cands_out),
                                    _stream(stream)))


def mc_classify(db: int, params: mc_classify_params, n_seq: int, seq, offs, n_queries: int, qoffs, label, hits,
                top_target=None, stream=None):
    _check(_lib.mc_classify(db, ctypes.byref(params), n_seq, _ptr(seq), _ptr(offs), n_queries, _ptr(qoffs),
                            _ptr(label), _ptr(hits), _ptr(top_target), _stream(stream)))


def mc_classify_debug(db: int, params: mc_classify_params, n_seq: int, seq, offs, n_queries: int, qoffs, label,
                      hits, top_target=None, cands=None, counters=None, stream=None):
    _check(_lib.mc_classify_debug(db, ctypes.byref(params), n_seq, _ptr(seq), _ptr(offs), n_queries, _ptr(qoffs),
                                  _ptr(label), _ptr(hits), _ptr(top_target), _ptr(cands), _ptr(counters),
                                  _stream(stream)))


MC_NOALLOC_MAX_QUERIES = 16384


def mc_classify_noalloc(db: int, params: mc_classify_params, n_seq: int, seq, offs, n_queries: int, qoffs, label,
                        hits, top_target=None, stream=None):
    """mc_classify without any device allocation (fixed scratch inside the
    library; at most MC_NOALLOC_MAX_QUERIES queries per call)."""
    _check(_lib.mc_classify_noalloc(db, ctypes.byref(params), n_seq, _ptr(seq), _ptr(offs), n_queries, _ptr(qoffs),
                                    _ptr(label), _ptr(hits), _ptr(top_target), _stream(stream)))


def mc_classify_status(db: int, stream=None):
    _check(_lib.mc_classify_status(db, _stream(stream)))


def mc_db_free(db: int):
    _lib.mc_db_free(db)


def mc_db_stats(db: int) -> dict:
    st = mc_db_stats_t()
    _check(_lib.mc_db_stats(db, ctypes.byref(st)))
    return {n: getattr(st, n) for n, _ in mc_db_stats_t._fields_}


def mc_db_dump(db: int, key_lo: int = 0, key_hi: int = 1 << 32):
    """(keys, counts, locs) of features in [key_lo, key_hi), ascending."""
    nk, nl = _u64(), _u64()
    code = _lib.mc_db_dump(db, key_lo, key_hi, 0, 0, None, None, None, ctypes.byref(nk), ctypes.byref(nl))
    if code not in (MC_OK, MC_ERR_CAPACITY):
        _check(code)
    if code == MC_ERR_CAPACITY and nk.value > 0:
        # sizes of locations are reported once the features fit
        code = _lib.mc_db_dump(db, key_lo, key_hi, nk.value, 0, None, None, None, ctypes.byref(nk),
                               ctypes.byref(nl))
        if code not in (MC_OK, MC_ERR_CAPACITY):
            _check(code)
    keys = np.zeros(max(1, nk.value), dtype=np.uint32)
    counts = np.zeros(max(1, nk.value), dtype=np.uint32)
    locs = np.zeros(max(1, nl.value), dtype=np.uint64)
    _check(_lib.mc_db_dump(db, key_lo, key_hi, nk.value, nl.value, keys.ctypes.data, counts.ctypes.data,
                           locs.ctypes.data, ctypes.byref(nk), ctypes.byref(nl)))
    return keys[:nk.value], counts[:nk.value], locs[:nl.value]


def mc_db_save(db: int, path: str):
    _check(_lib.mc_db_save(db, os.fsencode(path)))


def mc_db_load(path: str, stream=None) -> int:
    h = _vp()
    _check(_lib.mc_db_load(os.fsencode(path), _stream(stream), ctypes.byref(h)))
    return h.value


def mc_window_offsets(params: mc_db_params, n_seq: int, offs, win_offs, stream=None):
    _check(_lib.mc_window_offsets(ctypes.byref(params), n_seq, _ptr(offs), _ptr(win_offs), _stream(stream)))


def mc_sketch(params: mc_db_params, n_seq: int, seq, offs, win_offs, n_windows: int, sketch, counts, stream=None):
    _check(_lib.mc_sketch(ctypes.byref(params), n_seq, _ptr(seq), _ptr(offs), _ptr(win_offs), n_windows,
                          _ptr(sketch), _ptr(counts), _stream(stream)))


def tuning(**kw) -> mc_tuning:
    """mc_tuning from keyword arguments (missing fields = 0 = default)."""
    t = mc_tuning()
    for k, v in kw.items():
        setattr(t, k, int(v))
    return t


def batch(n_seq: int, seq, offs, qoffs, label, hits, top_target=None) -> mc_batch:
    """mc_batch descriptor of device tensors (n_queries = len(qoffs) - 1)."""
    n_q = (qoffs.numel() if hasattr(qoffs, "numel") else len(qoffs)) - 1
    return mc_batch(n_seq, n_q, _ptr(seq), _ptr(offs), _ptr(qoffs), _ptr(label), _ptr(hits), _ptr(top_target))


def _batch_array(batches):
    arr = (mc_batch * max(1, len(batches)))(*batches)
    return arr, len(batches)


def mc_db_set_tuning(db: int, t: mc_tuning | None):
    _check(_lib.mc_db_set_tuning(db, ctypes.byref(t) if t is not None else None))


def mc_classify_batches(db: int, params: mc_classify_params, batches, t: mc_tuning | None = None, stream=None):
    arr, n = _batch_array(batches)
    _check(_lib.mc_classify_batches(db, ctypes.byref(params), ctypes.byref(t) if t is not None else None, n, arr,
                                    _stream(stream)))


class Plan:
    """mc_plan: scratch + CUDA graph of one classify launch set, replayed by run()."""

    def __init__(self, db: int, params: mc_classify_params, max_batches: int, max_queries: int,
                 t: mc_tuning | None = None):
        h = _vp()
        _check(_lib.mc_plan_create(db, ctypes.byref(params), ctypes.byref(t) if t is not None else None,
                                   max_batches, max_queries, ctypes.byref(h)))
        self.handle = h.value

    def run(self, batches, stream=None):
        arr, n = _batch_array(batches)
        _check(_lib.mc_plan_run(self.handle, n, arr, _stream(stream)))

    @property
    def kernels(self) -> int:
        return _lib.mc_plan_kernels(self.handle)

    def free(self):
        if self.handle:
            _lib.mc_plan_free(self.handle)
            self.handle = 0


def mc_autotune(db: int, params: mc_classify_params, batches, reps: int = 3):
    """(best mc_tuning, [(stage, tuning dict, ms), ...]) on sample batches."""
    arr, n = _batch_array(batches)
    best = mc_tuning()
    times = (mc_tuning_time * 64)()
    nt = _u32()
    _check(_lib.mc_autotune(db, ctypes.byref(params), n, arr, reps, ctypes.byref(best), times, 64, ctypes.byref(nt)))
    rec = [(times[i].stage, times[i].tuning.as_dict(), float(times[i].ms)) for i in range(min(nt.value, 64))]
    return best, rec


class Server:
    """mc_server: a request loop over a resident database.  Jobs are host
    arrays (numpy or pinned torch tensors); their outputs are host arrays
    filled when wait() reports the job done."""

    def __init__(self, db: int, params: mc_classify_params, n_streams: int = 2, max_set_queries: int = 0,
                 max_set_jobs: int = 0, hbm_limit: int = 0):
        cfg = mc_server_config(n_streams, max_set_queries, max_set_jobs, 0, hbm_limit)
        h = _vp()
        _check(_lib.mc_server_create(db, ctypes.byref(params), ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h.value
        self._keep = {}

    def submit(self, n_seq: int, seq, offs, qoffs, label, hits, top_target=None) -> int:
        n_q = (qoffs.numel() if hasattr(qoffs, "numel") else len(qoffs)) - 1
        j = mc_job(n_seq, n_q, _ptr(seq), _ptr(offs), _ptr(qoffs), _ptr(label), _ptr(hits), _ptr(top_target))
        jid = _u64()
        _check(_lib.mc_server_submit(self.handle, ctypes.byref(j), ctypes.byref(jid)))
        self._keep[jid.value] = (seq, offs, qoffs, label, hits, top_target)
        return jid.value

    def extend(self, seq: np.ndarray, offs: np.ndarray, taxon: np.ndarray) -> int:
        seq = np.ascontiguousarray(seq, dtype=np.uint8)
        offs = np.ascontiguousarray(offs, dtype=np.uint64)
        taxon = np.ascontiguousarray(taxon, dtype=np.uint32)
        first = _u32()
        _check(_lib.mc_server_extend(self.handle, len(taxon), seq.ctypes.data, offs.ctypes.data, taxon.ctypes.data,
                                     ctypes.byref(first)))
        return first.value

    def wait(self, job_id: int, timeout: float = -1.0) -> dict | None:
        """Job info once done; None on timeout."""
        info = mc_job_info()
        code = _lib.mc_server_wait(self.handle, job_id, timeout, ctypes.byref(info))
        if code == MC_ERR_TIMEOUT:
            return None
        _check(code)
        self._keep.pop(job_id, None)
        return {n: getattr(info, n) for n, _ in mc_job_info._fields_}

    def drain(self, timeout: float = -1.0) -> bool:
        code = _lib.mc_server_drain(self.handle, timeout)
        if code == MC_ERR_TIMEOUT:
            return False
        _check(code)
        return True

    def stats(self) -> dict:
        st = mc_server_stats()
        _check(_lib.mc_server_stats_get(self.handle, ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in mc_server_stats._fields_}

    def free(self):
        if self.handle:
            _lib.mc_server_free(self.handle)
            self.handle = 0
            self._keep.clear()


def mc_debug_stall_next_sort(limit_ns: int):
    """Test export: the next database sort's last pass skips its first tile,
    so its bounded look-back wait gives up after limit_ns (MC_ERR_TIMEOUT)."""
    _check(_lib.mc_debug_stall_next_sort(limit_ns))


def mc_trace_enable(on: bool = True):
    _check(_lib.mc_trace_enable(int(on)))


def mc_trace_report(reset: bool = True) -> dict:
    """{kernel: (launches, total_ms)} of the traced launches since the last reset."""
    n = _lib.mc_trace_report(None, 0, 0)
    buf = ctypes.create_string_buffer(n + 1)
    _lib.mc_trace_report(buf, n + 1, int(reset))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def mc_kernel_launches() -> int:
    return int(_lib.mc_kernel_launches())


# ------------------------------------------------------- convenience layer
@dataclass
class Database:
    """Owning handle: create, add targets, finalize, classify, free."""
    handle: int
    params: mc_db_params

    @classmethod
    def create(cls, parent, stream=None, **params) -> "Database":
        p = db_params(**params)
        return cls(mc_db_create(p, len(parent), parent, stream), p)

    def add_targets(self, seq, offs, taxon) -> int:
        return mc_db_add_targets(self.handle, len(taxon), seq, offs, taxon)

    def finalize(self):
        mc_db_finalize(self.handle)

    def stats(self) -> dict:
        return mc_db_stats(self.handle)

    def save(self, path: str):
        mc_db_save(self.handle, path)

    @classmethod
    def load(cls, path: str, stream=None) -> "Database":
        return cls(mc_db_load(path, stream), None)

    def dump(self, lo=0, hi=1 << 32):
        return mc_db_dump(self.handle, lo, hi)

    def classify(self, seq, offs, qoffs, *, label=None, hits=None, top_target=None, cands=None, counters=None,
                 stream=None, **cparams):
        """Device tensors in, device tensors out: (label, hits, top_target[, cands])."""
        import torch
        nq = qoffs.numel() - 1
        dev = seq.device
        label = torch.empty(nq, dtype=torch.int32, device=dev) if label is None else label
        hits = torch.empty(nq, dtype=torch.int32, device=dev) if hits is None else hits
        top_target = torch.empty(nq, dtype=torch.int32, device=dev) if top_target is None else top_target
        cp = classify_params(**cparams)
        mc_classify_debug(self.handle, cp, offs.numel() - 1, seq, offs, nq, qoffs, label, hits, top_target, cands,
                          counters, stream)
        return label, hits, top_target

    def free(self):
        if self.handle:
            mc_db_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
