"""CPU oracle for the dense Pauli decomposition -- TEST INFRASTRUCTURE, not the product.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package. It shares no code with the CUDA library and never imports it.

Two independent formulations, both plain and slow:

* ``decompose_at`` / ``compose_at``: the C routines in ``pauli_oracle.c`` -- Eq. (13) with
  the per-digit lambda of Eq. (12), and Eq. (1) with the element product of Eq. (7),
  Neumaier-compensated FP64 sums, OpenMP over the requested outputs.
* ``kron``: explicit Pauli tensors built by Kronecker products of the matrices of Eq. (3),
  and the trace of Eq. (4), in NumPy (used for N <= 4).
* ``weighted_norm`` / ``weighted_norm_grad``: the real loss sum_n w_n |c_n|^2 of the adjoint
  workload and its gradient 2 w c, by their definitions, in NumPy.

Precision: FP64. A complex64 input is upcast exactly to complex128 before the call, so the
oracle value for a complex64 input is the exact-input FP64 result.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

from . import kron  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pauli_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile pauli_oracle.c into liboracle.so with gcc (OpenMP, no fast-math), and the
    Gray-code CPU baseline (``oracle.gray``) beside it."""
    from . import gray

    gray.build(force)
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
            u64p = ctypes.POINTER(ctypes.c_uint64)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_decompose_at.argtypes = [dp, ctypes.c_int, u64p, ctypes.c_int64, dp, ctypes.c_int]
            lib.oracle_decompose_at.restype = ctypes.c_int
            lib.oracle_compose_at.argtypes = [dp, ctypes.c_int, u64p, u64p, ctypes.c_int64, dp, ctypes.c_int]
            lib.oracle_compose_at.restype = ctypes.c_int
            lib.oracle_default_threads.argtypes = []
            lib.oracle_default_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def default_threads() -> int:
    """Threads the oracle uses when none are requested (OpenMP default)."""
    return int(_load().oracle_default_threads())


def _as_c128(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a).astype(np.complex128, copy=False))


def _nqubits(G: np.ndarray) -> int:
    D = G.shape[-1]
    if G.ndim != 2 or G.shape[0] != D or D < 2 or (D & (D - 1)):
        raise ValueError("G must be a square 2^N x 2^N matrix")
    return D.bit_length() - 1


def decompose_at(G: np.ndarray, idx, threads: int = 0) -> np.ndarray:
    """c_n for each n in ``idx`` by Eq. (13) (complex128)."""
    G = _as_c128(G)
    N = _nqubits(G)
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.uint64).ravel())
    out = np.empty(idx.size, dtype=np.complex128)
    lib = _load()
    rc = lib.oracle_decompose_at(G.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), N,
                                 idx.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), idx.size,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(threads))
    if rc != 0:
        raise ValueError("oracle_decompose_at rejected its arguments")
    return out


def decompose_full(G: np.ndarray, threads: int = 0) -> np.ndarray:
    """All 4^N coefficients, in the paper's order n."""
    N = _nqubits(np.asarray(G))
    return decompose_at(G, np.arange(4 ** N, dtype=np.uint64), threads)


def compose_at(c: np.ndarray, rows, cols, threads: int = 0) -> np.ndarray:
    """[sum_n c_n P_n]_{rows[q], cols[q]} by Eqs. (1) and (7)."""
    c = _as_c128(c).ravel()
    nc = c.size
    N = (nc.bit_length() - 1) // 2
    if nc < 4 or 4 ** N != nc:
        raise ValueError("c must hold 4^N coefficients")
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.uint64).ravel())
    cols = np.ascontiguousarray(np.asarray(cols, dtype=np.uint64).ravel())
    if rows.size != cols.size:
        raise ValueError("rows and cols differ in length")
    out = np.empty(rows.size, dtype=np.complex128)
    lib = _load()
    rc = lib.oracle_compose_at(c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), N,
                               rows.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                               cols.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), rows.size,
                               out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(threads))
    if rc != 0:
        raise ValueError("oracle_compose_at rejected its arguments")
    return out


def compose_full(c: np.ndarray, threads: int = 0) -> np.ndarray:
    """G = sum_n c_n P_n as a dense 2^N x 2^N complex128 matrix."""
    c = np.asarray(c).ravel()
    N = (c.size.bit_length() - 1) // 2
    D = 1 << N
    r, q = np.divmod(np.arange(D * D, dtype=np.uint64), np.uint64(D))
    return compose_at(c, r, q, threads).reshape(D, D)


def decompose_grad(grad_c: np.ndarray, threads: int = 0) -> np.ndarray:
    """Gradient of a real loss with respect to G, given torch's grad with respect to c.

    c = A vec(G) with A[n, (j, i)] = 2^-N [P_n]_{ij}. Under the conjugate-Wirtinger
    convention the gradient of a linear map is A^H grad_c, and since every P_n is
    Hermitian this is 2^-N sum_n grad_c[n] P_n = 2^-N compose(grad_c).
    """
    grad_c = np.asarray(grad_c).ravel()
    N = (grad_c.size.bit_length() - 1) // 2
    return compose_full(grad_c, threads) * (2.0 ** -N)


def weighted_norm(c: np.ndarray, w: np.ndarray) -> float:
    """sum_k sum_n w_n |c_{k,n}|^2 for coefficient vectors along the last axis of c.

    The real loss of the adjoint workload. Each term in FP64 from the exactly upcast input,
    the terms added with math.fsum (correctly rounded sum of the rounded terms).
    """
    c = _as_c128(c)
    w = np.asarray(w, dtype=np.float64)
    if c.shape[-1] != w.size:
        raise ValueError("w must hold one weight per coefficient index")
    terms = w * (c.real * c.real + c.imag * c.imag)
    return math.fsum(terms.ravel().tolist())


def weighted_norm_grad(c: np.ndarray, w: np.ndarray, g: float = 1.0) -> np.ndarray:
    """g times the gradient of weighted_norm in torch's convention for complex inputs:
    dL/dRe c + i dL/dIm c = 2 w_n c_{k,n}, in FP64."""
    c = _as_c128(c)
    w = np.asarray(w, dtype=np.float64)
    if c.shape[-1] != w.size:
        raise ValueError("w must hold one weight per coefficient index")
    return (2.0 * g * w) * c


def y_count(idx, N: int) -> np.ndarray:
    """Number of Y factors of P_n for each n: base-4 digits of n equal to 2 (Eq. (2): digit t of n
    names operator t as I, X, Y, Z for 0..3)."""
    n = np.asarray(idx, dtype=np.uint64).ravel()
    k = np.zeros(n.shape, dtype=np.int64)
    for t in range(N):
        k += ((n >> np.uint64(2 * t)) & np.uint64(3)) == 2
    return k


def real_coefficients_at(G_real: np.ndarray, idx) -> np.ndarray:
    """For a real matrix G: the real a_n with c_n = i^(k mod 2) a_n, k = y_count(n) (c_n is real
    for even k and imaginary for odd k, since every Y entry is imaginary, Eq. (3)). Computed as
    c_n (decompose_at of G + 0i) times (-i)^(k mod 2); the discarded part is exactly zero."""
    G = np.asarray(G_real, dtype=np.float64)
    N = _nqubits(G)
    c = decompose_at(G.astype(np.complex128), idx)
    k = y_count(idx, N)
    return np.where(k % 2 == 1, (c * -1j).real, c.real)
