"""The oracle's pins have teeth: plausible mistakes planted in a copy of the oracle's C source
(on the CPU, in a temporary directory) must each fail at least one pin."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg

from oracle import kron
from paper_2401_16378_gb300 import workloads

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "pauli_oracle.c")

MUTANTS = {
    "y_sign_flipped": ("{{{0.0, 0.0}, {0.0, -1.0}}, {{0.0, 1.0}, {0.0, 0.0}}}",
                       "{{{0.0, 0.0}, {0.0, 1.0}}, {{0.0, -1.0}, {0.0, 0.0}}}"),
    "row_col_transposed": ("G + 2 * ((i ^ m) * D + i)", "G + 2 * (i * D + (i ^ m))"),
    "scale_dropped": ("out[0] = nsum_value(&sr) * scale;", "out[0] = nsum_value(&sr);"),
    "digit_bits_swapped": ("return (bit_of(n, 2 * t + 1) << 1) | bit_of(n, 2 * t);",
                           "return (bit_of(n, 2 * t) << 1) | bit_of(n, 2 * t + 1);"),
    "xy_mask_wrong": ("if (p == 1u || p == 2u)", "if (p == 1u || p == 3u)"),
    "lambda_column_wrong": ("unsigned b = a ^ bit_of(m, t);", "unsigned b = a;"),
    "imag_term_sign": ("nsum_add(&si, lr * g[1] + li * g[0]);", "nsum_add(&si, lr * g[1] - li * g[0]);"),
    # the compensated sum: its value without the compensation, the branch for the larger
    # running sum using the other branch's formula, a plain running sum, and the composition
    # returning its sums without their compensation
    "neumaier_value_drops_comp": ("return a->sum + a->comp;", "return a->sum;"),
    "neumaier_branch_swapped": ("a->comp += (a->sum - t) + x;\n  else", "a->comp += (x - t) + a->sum;\n  else"),
    "neumaier_plain_sum": ("double t = a->sum + x;\n", "double t = a->sum + x;\n  a->sum = t;\n  return;\n"),
    "compose_compensation_dropped": ("out[0] = nsum_value(&sr);\n  out[1] = nsum_value(&si);",
                                     "out[0] = sr.sum;\n  out[1] = si.sum;"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation anchor for {name} not found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new, 1))
    lib = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", str(lib), str(path), "-lm"],
                   check=True)
    L = ctypes.CDLL(str(lib))
    dp = ctypes.POINTER(ctypes.c_double)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.oracle_decompose_at.argtypes = [dp, ctypes.c_int, u64p, ctypes.c_int64, dp, ctypes.c_int]
    L.oracle_decompose_at.restype = ctypes.c_int
    L.oracle_compose_at.argtypes = [dp, ctypes.c_int, u64p, u64p, ctypes.c_int64, dp, ctypes.c_int]
    L.oracle_compose_at.restype = ctypes.c_int

    def decompose_full(G):
        G = np.ascontiguousarray(G, dtype=np.complex128)
        N = G.shape[0].bit_length() - 1
        idx = np.arange(4 ** N, dtype=np.uint64)
        out = np.empty(idx.size, dtype=np.complex128)
        rc = L.oracle_decompose_at(G.ctypes.data_as(dp), N, idx.ctypes.data_as(u64p), idx.size,
                                   out.ctypes.data_as(dp), 1)
        assert rc == 0
        return out

    def compose_diag(c):
        c = np.ascontiguousarray(c, dtype=np.complex128)
        N = (c.size.bit_length() - 1) // 2
        r = np.arange(1 << N, dtype=np.uint64)
        out = np.empty(r.size, dtype=np.complex128)
        rc = L.oracle_compose_at(c.ctypes.data_as(dp), N, r.ctypes.data_as(u64p), r.ctypes.data_as(u64p), r.size,
                                 out.ctypes.data_as(dp), 1)
        assert rc == 0
        return out

    return decompose_full, compose_diag


def _compensation_pins_pass(decompose_full, compose_diag):
    """The exact cancelling-diagonal pins of test_oracle.py at N = 6 (Eqs. (13) and (1))."""
    N, D, big = 6, 64, 2 ** 60
    rng = np.random.default_rng(5)
    d = rng.integers(-5, 6, size=D).astype(np.int64)
    d[0], d[-1] = big, -big
    H = scipy.linalg.hadamard(D, dtype=np.int64)
    exact = np.array([float(int(v)) for v in H @ d])
    zidx = np.array([sum(3 << (2 * t) for t in range(N) if (z >> t) & 1) for z in range(D)])
    G = np.diag(d.astype(np.float64)).astype(np.complex128)
    if not np.array_equal(decompose_full(G)[zidx].real, exact * 2.0 ** -N):
        return False
    c = np.zeros(4 ** N, dtype=np.complex128)
    c[zidx] = d.astype(np.float64)
    return np.array_equal(compose_diag(c).real, exact)


def _pins_pass(fns):
    decompose_full, compose_diag = fns
    if not _compensation_pins_pass(decompose_full, compose_diag):
        return False
    G1 = np.array([[1, 2], [3, 4]], dtype=np.complex128)
    if not np.array_equal(decompose_full(G1), np.array([2.5, 2.5, -0.5j, -1.5])):
        return False
    for n in (1, 2, 3, 4, 15):
        c = decompose_full(kron.pauli_tensor(n, 2))
        if not (c[n] == 1 and np.count_nonzero(c) == 1):
            return False
    G = workloads.gaussian_complex(3, 77)
    return np.allclose(decompose_full(G), kron.decompose(G), rtol=0, atol=1e-13)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not found")
def test_unmutated_copy_passes(tmp_path):
    assert _pins_pass(_build(tmp_path, "identity", "#include <math.h>", "#include <math.h>"))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc not found")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _pins_pass(_build(tmp_path, name, old, new))
