"""Seeded synthetic inputs for the Pauli decomposition workloads.

This module only draws random numbers; it holds none of the decomposition's arithmetic and
imports neither the CUDA binding nor the oracle, so both sides of every parity check can use
it. The paper benchmarks on random dense complex matrices (Sec. 4); there is no dataset.

Recipe (NumPy ``default_rng(seed)``; complex entries have real and imaginary parts i.i.d.
standard normal, the whole real part drawn first, row by row, then the whole imaginary part):

* ``n6``       N=6, seed 0, all 4^6 coefficients.
* ``n12``      N=12, seed 12 (general) and seed 1012 (Hermitian (A + A^H)/2); 4096 sampled
               coefficient indices from seed 12012 plus the special indices below.
* ``n14``      N=14, seed 14 (4 GiB complex128; complex64 = the rounded cast of it);
               4096 sampled indices from seed 14014 plus the special indices.
* ``batched``  seed 512: N_b = integers(3, 11, 512) (3..10 inclusive), then for each b in
               order A_b complex normal, G_b = (A_b + A_b^H)/2.
* ``adjoint``  seed 64: 64 complex normal 1024 x 1024 matrices; weights w_n from seed 6464,
               uniform(0, 1), one vector of length 4^10 shared by the batch; gradcheck at N=4
               with seed 4.

Special coefficient indices: 0 (all identity), 1, 2, 3, all-X (every base-4 digit 1),
all-Y (every digit 2) and all-Z (every digit 3, which is 4^N - 1).
"""
from __future__ import annotations

import numpy as np

SEEDS = {"n6": 0, "n12": 12, "n12_herm": 1012, "n12_idx": 12012, "n14": 14, "n14_idx": 14014,
         "batched": 512, "adjoint": 64, "adjoint_w": 6464, "gradcheck": 4}

_ROW_CHUNK = 1024


def _fill_normal(rng: np.random.Generator, out: np.ndarray) -> None:
    """Fill ``out`` (2-D float64) with standard normals in row-major order, in row chunks."""
    for r in range(0, out.shape[0], _ROW_CHUNK):
        rng.standard_normal(out=out[r:r + _ROW_CHUNK])


def gaussian_complex(N: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """2^N x 2^N matrix with real and imaginary parts i.i.d. N(0, 1)."""
    D = 1 << N
    rng = np.random.default_rng(seed)
    G = np.empty((D, D), dtype=np.complex128)
    part = np.empty((min(D, _ROW_CHUNK), D), dtype=np.float64)
    for which in ("real", "imag"):
        for r in range(0, D, _ROW_CHUNK):
            blk = part[: min(_ROW_CHUNK, D - r)]
            rng.standard_normal(out=blk)
            getattr(G[r:r + blk.shape[0]], which)[...] = blk
    return G if dtype == np.complex128 else G.astype(dtype)


def hermitian_from(A: np.ndarray) -> np.ndarray:
    """(A + A^H) / 2 -- the Hermitian part of A."""
    return (A + A.conj().T) * 0.5


def hermitian_complex(N: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """(A + A^H)/2 with A = gaussian_complex(N, seed)."""
    G = hermitian_from(gaussian_complex(N, seed))
    return G if dtype == np.complex128 else G.astype(dtype)


def integer_complex(N: int, seed: int, lo: int = -8, hi: int = 8, dtype=np.complex128) -> np.ndarray:
    """Integer-valued entries in [lo, hi] for both parts (sums of these are exact in FP64)."""
    D = 1 << N
    rng = np.random.default_rng(seed)
    re = rng.integers(lo, hi + 1, size=(D, D)).astype(np.float64)
    im = rng.integers(lo, hi + 1, size=(D, D)).astype(np.float64)
    return (re + 1j * im).astype(dtype)


def gaussian_coefficients(N: int, seed: int, dtype=np.complex128) -> np.ndarray:
    """4^N complex coefficients with real and imaginary parts i.i.d. N(0, 1) (real part first)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(4 ** N)
    im = rng.standard_normal(4 ** N)
    return (re + 1j * im).astype(dtype)


def special_indices(N: int) -> np.ndarray:
    """0, 1, 2, 3, all-X, all-Y, all-Z coefficient indices (deduplicated, sorted)."""
    all_x = sum(1 << (2 * t) for t in range(N))
    idx = {0, 1, 2, 3, all_x, 2 * all_x, 3 * all_x}
    return np.array(sorted(i for i in idx if i < 4 ** N), dtype=np.uint64)


def sample_indices(N: int, seed: int, k: int = 4096, with_special: bool = True) -> np.ndarray:
    """k seeded random coefficient indices in [0, 4^N), then the special indices appended."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, 4 ** N, size=k, dtype=np.uint64)
    if with_special:
        idx = np.concatenate([idx, special_indices(N)])
    return idx


def batched_hermitian(seed: int = 512, batch: int = 512, nmin: int = 3, nmax: int = 10,
                      dtype=np.complex128) -> tuple[list[np.ndarray], np.ndarray]:
    """The uneven-N Hermitian batch: returns (list of matrices, array of N)."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(nmin, nmax + 1, size=batch)
    mats = []
    for N in Ns:
        D = 1 << int(N)
        A = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
        mats.append(hermitian_from(A).astype(dtype))
    return mats, Ns.astype(np.int64)


def adjoint_inputs(seed: int = 64, batch: int = 64, N: int = 10, dtype=np.complex128) -> np.ndarray:
    """(batch, 2^N, 2^N) complex normal matrices for the adjoint workload."""
    D = 1 << N
    rng = np.random.default_rng(seed)
    out = np.empty((batch, D, D), dtype=np.complex128)
    for b in range(batch):
        out[b].real = rng.standard_normal((D, D))
        out[b].imag = rng.standard_normal((D, D))
    return out if dtype == np.complex128 else out.astype(dtype)


def adjoint_weights(seed: int = 6464, N: int = 10) -> np.ndarray:
    """w_n ~ U(0, 1), length 4^N."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=4 ** N)
