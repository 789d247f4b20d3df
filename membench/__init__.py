"""Random-access read bandwidth of the GPU, for the benchmark's roofline.

The classification kernels probe the feature table and gather buckets with
16-32 byte reads at random positions, which HBM serves far below its copy
bandwidth.  `random_read_gbs` measures that rate on the current device
(membench.cu, built into libmembench.so next to it).  It is a measurement
aid of bench.py, not part of the classification library.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "membench.cu")
_LIB = os.path.join(_HERE, "libmembench.so")
_lib = None


def _nvcc() -> str:
    for c in [os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"]:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmembench.so")


def build(force: bool = False) -> str:
    """Compile membench.cu for sm_103a into libmembench.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo",
                               "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, _SRC])
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
