"""Randomised pins of the oracle (hypothesis, CPU): symmetries of the Pauli basis that a dropped
sign, a swapped index or a transposed operand would break. Integer-valued inputs keep every
sum exact, so the identities hold bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import kron

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings


@st.composite
def int_matrix(draw, max_n=3):
    N = draw(st.integers(1, max_n))
    D = 1 << N
    re = draw(st.lists(st.integers(-4, 4), min_size=D * D, max_size=D * D))
    im = draw(st.lists(st.integers(-4, 4), min_size=D * D, max_size=D * D))
    return N, (np.array(re, dtype=float) + 1j * np.array(im, dtype=float)).reshape(D, D)


def _digits(n, N):
    return [(n >> (2 * t)) & 3 for t in range(N)]


def _anticommute_sign(m, n, N):
    """(-1)^s with s the number of factors where P_m and P_n are different non-identity Paulis."""
    s = sum(1 for a, b in zip(_digits(m, N), _digits(n, N)) if a and b and a != b)
    return -1 if s % 2 else 1


@settings(max_examples=30, deadline=None)
@given(int_matrix())
def test_conjugate_transpose_conjugates_coefficients(arg):
    """Every P_n is Hermitian: c_n(G^H) = conj(c_n(G))."""
    N, G = arg
    np.testing.assert_array_equal(oracle.decompose_full(G.conj().T), np.conj(oracle.decompose_full(G)))


@settings(max_examples=30, deadline=None)
@given(int_matrix())
def test_transpose_flips_sign_of_odd_y_strings(arg):
    """Y^T = -Y and X, Z, I are symmetric: c_n(G^T) = (-1)^(number of Y factors) c_n(G)."""
    N, G = arg
    k = oracle.y_count(range(4 ** N), N)
    np.testing.assert_array_equal(oracle.decompose_full(G.T), np.where(k % 2 == 1, -1, 1) * oracle.decompose_full(G))


@settings(max_examples=20, deadline=None)
@given(int_matrix(max_n=2), st.integers(0, 15))
def test_pauli_conjugation_signs(arg, m):
    """c_n(P_m G P_m) = (-1)^[P_m and P_n anticommute] c_n(G)."""
    N, G = arg
    m = m % (4 ** N)
    P = kron.pauli_tensor(m, N)
    got = oracle.decompose_full(P @ G @ P)
    want = np.array([_anticommute_sign(m, n, N) for n in range(4 ** N)]) * oracle.decompose_full(G)
    np.testing.assert_array_equal(got, want)


@settings(max_examples=20, deadline=None)
@given(int_matrix(), st.integers(-3, 3), st.integers(-3, 3))
def test_linearity_and_exact_reconstruction(arg, a, b):
    N, G = arg
    H = np.roll(G, 1, axis=0) - 2j * G.T
    ca, cb = oracle.decompose_full(G), oracle.decompose_full(H)
    np.testing.assert_array_equal(oracle.decompose_full(a * G + b * H), a * ca + b * cb)
    np.testing.assert_array_equal(oracle.compose_full(ca), G)
