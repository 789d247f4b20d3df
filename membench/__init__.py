"""Measurement aids of bench.py (libmembench.so), not part of the
classification library.

- `random_read_gbs`: random-access read bandwidth of the GPU, for the
  benchmark's roofline.  The classification kernels probe the feature table
  and gather buckets with 16-32 byte reads at random positions, which HBM
  serves far below its copy bandwidth (membench.cu).
- `hash_insert_build`: the paper's build primitive, every (feature,
  location) pair inserted into a hash table with warp-aggregated atomics
  (insertbench.cu), timed on the same pairs as the library's sort-based
  build.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "membench.cu")
_SRC_INSERT = os.path.join(_HERE, "insertbench.cu")
_LIB = os.path.join(_HERE, "libmembench.so")
_lib = None


def _nvcc() -> str:
    for c in [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmembench.so")


def build(force: bool = False) -> str:
    """Compile membench.cu for sm_103a into libmembench.so."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_INSERT))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
                               "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _SRC, _SRC_INSERT])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB):
            raise ImportError(f"{_LIB} is missing: run membench.build()")
        lib = ctypes.CDLL(_LIB)
        lib.membench_random_read.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p,
                                             ctypes.POINTER(ctypes.c_double)]
        lib.membench_random_read.restype = ctypes.c_int
        lib.membench_last_error.restype = ctypes.c_char_p
        u32, u64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
        pd = ctypes.POINTER(ctypes.c_double)
        lib.membench_insert_count.argtypes = [vp, vp, u64, u32, u32, u32, vp, vp, vp, vp, pd]
        lib.membench_insert_count.restype = ctypes.c_int
        lib.membench_insert_fill.argtypes = [vp, vp, u64, u32, u32, u32, vp, vp, vp, vp, u32, vp, vp, pd]
        lib.membench_insert_fill.restype = ctypes.c_int
        lib.membench_insert_last_error.restype = ctypes.c_char_p
        _lib = lib
    return _lib


def random_read_gbs(buf_bytes: int, width: int, n_reads: int, stream: int | None = None) -> float:
    """GB/s of `width`-byte reads (16 or 32) at random positions of a fresh
    buf_bytes device buffer (best of several launch shapes).  `stream` is a
    cudaStream_t value (None = the legacy stream)."""
    lib = _load()
    v = ctypes.c_double()
    rc = lib.membench_random_read(buf_bytes, width, n_reads, stream, ctypes.byref(v))
    if rc != 0:
        raise ValueError(lib.membench_last_error().decode()) if rc == 1 else \
            RuntimeError(lib.membench_last_error().decode())
    return v.value


def _insert_check(lib, rc: int):
    if rc != 0:
        msg = lib.membench_insert_last_error().decode()
        raise ValueError(msg) if rc == 1 else RuntimeError(msg)


def hash_insert_build(sketch, counts, n_windows: int, s: int, cap: int, log_slots: int, stream=None,
                      max_probe: int = 4096, return_tables: bool = False) -> dict:
    """The paper's build primitive, timed: every (feature, window) pair of
    the window sketches (device tensors: sketch int32[n_windows * s],
    counts int32[n_windows], as mc_sketch writes them) inserted into a hash
    table of 2^log_slots slots with warp-aggregated atomics, at most `cap`
    locations per feature (insertbench.cu).  Passes: count, exclusive scan
    of min(count, cap) (torch), fill.  Returns their times in ms (CUDA
    events on `stream`, default the current torch stream) and the table's
    distinct features and kept locations (with return_tables, also the
    device tensors keys, count, offset and vals)."""
    import torch
    lib = _load()
    dev = sketch.device
    st = torch.cuda.current_stream(dev) if stream is None else stream
    handle = ctypes.c_void_p(st.cuda_stream)
    slots = 1 << log_slots
    keys = torch.full((slots,), -1, dtype=torch.int32, device=dev)
    cnt = torch.zeros(slots, dtype=torch.int32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    ms_count, ms_fill = ctypes.c_double(), ctypes.c_double()
    torch.cuda.synchronize(dev)
    _insert_check(lib, lib.membench_insert_count(sketch.data_ptr(), counts.data_ptr(), n_windows, s, log_slots,
                                                 max_probe, keys.data_ptr(), cnt.data_ptr(), err.data_ptr(), handle,
                                                 ctypes.byref(ms_count)))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        a.record()
        capped = torch.clamp(cnt, max=cap).to(torch.int64)
        offset = torch.cumsum(capped, 0)
        n_kept = int(offset[-1].item()) if slots else 0
        offset -= capped
        b.record()
    b.synchronize()
    ms_scan = a.elapsed_time(b)
    del capped
    cursor = torch.zeros(slots, dtype=torch.int32, device=dev)
    vals = torch.empty(max(1, n_kept), dtype=torch.int32, device=dev)
    _insert_check(lib, lib.membench_insert_fill(sketch.data_ptr(), counts.data_ptr(), n_windows, s, log_slots,
                                                max_probe, keys.data_ptr(), offset.data_ptr(), cursor.data_ptr(),
                                                vals.data_ptr(), cap, err.data_ptr(), handle, ctypes.byref(ms_fill)))
    n_keys = int((keys != -1).sum().item())
    out = {"count_ms": round(ms_count.value, 3), "scan_ms": round(ms_scan, 3), "fill_ms": round(ms_fill.value, 3),
           "total_ms": round(ms_count.value + ms_scan + ms_fill.value, 3), "n_keys": n_keys, "n_kept": n_kept,
           "slots": slots}
    if return_tables:
        out["tables"] = {"keys": keys, "count": cnt, "offset": offset, "vals": vals}
    return out
