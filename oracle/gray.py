"""The paper's Gray-code algorithm on the CPU (Sec. 3, Eq. (14); C + OpenMP in gray_baseline.c).

A faster CPU baseline for the benchmark, not the checker: the tests hold it to the oracle
(``oracle.decompose_at``). Same conventions and the same call shape as ``decompose_at``; plain
FP64 sums.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gray_baseline.c")
_LIB_PATH = os.path.join(_HERE, "libgray.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gray_baseline.c into libgray.so (gcc, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.gray_decompose_at.argtypes = [dp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int64,
                                              dp, ctypes.c_int]
            lib.gray_decompose_at.restype = ctypes.c_int
            lib.gray_default_threads.argtypes = []
            lib.gray_default_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def default_threads() -> int:
    return int(_load().gray_default_threads())


def decompose_at(G: np.ndarray, idx, threads: int = 0) -> np.ndarray:
    """c_n for each n in ``idx`` by the Gray-code recurrence (complex128)."""
    G = np.ascontiguousarray(np.asarray(G).astype(np.complex128, copy=False))
    D = G.shape[-1]
    if G.ndim != 2 or G.shape[0] != D or D < 2 or (D & (D - 1)):
        raise ValueError("G must be a square 2^N x 2^N matrix")
    N = D.bit_length() - 1
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64).ravel())
    out = np.empty(idx.size, dtype=np.complex128)
    rc = _load().gray_decompose_at(G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), N,
                                   idx.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), idx.size,
                                   out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(threads))
    if rc != 0:
        raise ValueError("gray_decompose_at rejected its arguments")
    return out
