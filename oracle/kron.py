"""Explicit Pauli tensors and the trace definition, in NumPy (oracle, test infrastructure).

This is a second, independent formulation of the decomposition for small N (N <= 4):

* The Pauli matrices are those of Eq. (3).
* P_n is the Kronecker product sigma_{N-1} (x) ... (x) sigma_0 (Eq. (6)), where operator t is
  the t-th base-4 digit of n (Sec. 2, last paragraph) and operator 0 is the rightmost factor
  (Sec. 2, first paragraph; Eq. (2): c_1 multiplies 1 (x) X, c_4 multiplies X (x) 1).
* c_n = 2^-N Tr(P_n G) (Eq. (4)), evaluated with a dense matrix product.
"""
from __future__ import annotations

import numpy as np

I2 = np.array([[1, 0], [0, 1]], dtype=np.complex128)
X2 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z2 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULIS = (I2, X2, Y2, Z2)
LABELS = "IXYZ"


def digits(n: int, N: int) -> list[int]:
    """Base-4 digits of n, operator 0 first."""
    return [(n >> (2 * t)) & 3 for t in range(N)]


def label(n: int, N: int) -> str:
    """Pauli string of tensor n, written leftmost factor first (operator N-1 ... 0)."""
    return "".join(LABELS[d] for d in reversed(digits(n, N)))


def pauli_tensor(n: int, N: int) -> np.ndarray:
    """P_n as a dense 2^N x 2^N matrix, built by Kronecker products (Eq. (6))."""
    P = np.ones((1, 1), dtype=np.complex128)
    for d in reversed(digits(n, N)):  # leftmost factor is operator N-1
        P = np.kron(P, PAULIS[d])
    return P


def decompose(G: np.ndarray) -> np.ndarray:
    """All 4^N coefficients by c_n = 2^-N Tr(P_n G) (Eq. (4))."""
    G = np.asarray(G, dtype=np.complex128)
    D = G.shape[0]
    N = D.bit_length() - 1
    return np.array([np.trace(pauli_tensor(n, N) @ G) / D for n in range(4 ** N)])


def compose(c: np.ndarray) -> np.ndarray:
    """G = sum_n c_n P_n (Eq. (1))."""
    c = np.asarray(c, dtype=np.complex128).ravel()
    N = (c.size.bit_length() - 1) // 2
    D = 1 << N
    G = np.zeros((D, D), dtype=np.complex128)
    for n in range(c.size):
        G += c[n] * pauli_tensor(n, N)
    return G
