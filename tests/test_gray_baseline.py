"""The Gray-code CPU baseline (the paper's Sec. 3 algorithm with the recurrence of Eq. (14)),
held to the oracle: every coefficient for small N, exactly on integer-valued inputs, sampled
coefficients at N = 10, and one-hot results for single Pauli tensors."""
import numpy as np
import pytest

import oracle
from oracle import gray, kron
from paper_2401_16378_gb300 import workloads


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6])
def test_matches_the_oracle_everywhere(N):
    G = workloads.gaussian_complex(N, 60 + N)
    idx = np.arange(4 ** N, dtype=np.uint64)
    err = np.max(np.abs(gray.decompose_at(G, idx) - oracle.decompose_at(G, idx)))
    assert err <= 1e-14 * np.max(np.abs(G))


def test_exact_on_integer_inputs():
    rng = np.random.default_rng(70)
    N = 5
    D = 1 << N
    G = (rng.integers(-8, 9, (D, D)) + 1j * rng.integers(-8, 9, (D, D))).astype(np.complex128)
    idx = np.arange(4 ** N, dtype=np.uint64)
    np.testing.assert_array_equal(gray.decompose_at(G, idx), oracle.decompose_at(G, idx))


def test_sampled_coefficients_at_n10():
    G = workloads.gaussian_complex(10, 71)
    idx = workloads.sample_indices(10, 72, k=256)
    err = np.max(np.abs(gray.decompose_at(G, idx, threads=2) - oracle.decompose_at(G, idx)))
    assert err <= 1e-13 * np.max(np.abs(G))


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4 * 2 + 3, 39, 63])
def test_single_pauli_tensor_is_one_hot(n):
    N = 3
    P = kron.pauli_tensor(n, N)
    c = gray.decompose_at(P, np.arange(4 ** N, dtype=np.uint64))
    want = np.zeros(4 ** N, dtype=np.complex128)
    want[n] = 1.0
    np.testing.assert_array_equal(c, want)


def test_rejects_out_of_range_indices():
    G = workloads.gaussian_complex(2, 73)
    with pytest.raises(ValueError):
        gray.decompose_at(G, np.array([16], dtype=np.uint64))
