"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: the paper's printed ordering and
matrices (tests/golden), hand-derived closed forms, exact integer arithmetic, an explicit
Kronecker-product formulation of the trace, library routines (scipy's Sylvester Hadamard
matrix), invariants of the Pauli basis, and a restatement of the paper's Gray-code variant.
"""
import ast
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
from oracle import kron
from paper_2401_16378_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(N, seed):
    return workloads.gaussian_complex(N, seed)


def test_threads_positive():
    assert oracle.default_threads() >= 1


def test_pauli_matrices_fixture():
    """Eq. (3): the four Pauli matrices used by both oracle formulations."""
    rows = {}
    with open(os.path.join(GOLDEN, "pauli_matrices.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            rows[name] = np.array([complex(ast.literal_eval(v)) for v in vals]).reshape(2, 2)
    for name, P in zip("IXYZ", kron.PAULIS):
        np.testing.assert_array_equal(P, rows[name])
        # the C oracle decomposes each Pauli matrix into a one-hot vector
        c = oracle.decompose_full(rows[name])
        np.testing.assert_array_equal(c, np.eye(4)["IXYZ".index(name)])


def test_eq2_ordering_fixture():
    """Eq. (2): c_1 multiplies 1(x)X, c_4 multiplies X(x)1, c_15 multiplies Z(x)Z, ..."""
    with open(os.path.join(GOLDEN, "eq2_ordering_n2.txt")) as f:
        pairs = [line.split() for line in f if line.strip() and not line.startswith("#")]
    assert len(pairs) == 6
    P = dict(zip("IXYZ", kron.PAULIS))
    for n_str, lab in pairs:
        n = int(n_str)
        assert kron.label(n, 2) == lab
        explicit = np.kron(P[lab[0]], P[lab[1]])  # leftmost factor first
        np.testing.assert_array_equal(kron.pauli_tensor(n, 2), explicit)
        c = oracle.decompose_full(explicit)
        expect = np.zeros(16)
        expect[n] = 1
        np.testing.assert_array_equal(c, expect)


def test_one_qubit_closed_form():
    """Eq. (4) at N=1 by hand: c_I=(g00+g11)/2, c_X=(g01+g10)/2, c_Y=i(g01-g10)/2, c_Z=(g00-g11)/2.

    For G = [[1, 2], [3, 4]]: Tr(Y G) = (-i)(3) + (i)(2) = -i, so c_Y = -0.5i, and
    c = (2.5, 2.5, -0.5i, -1.5).
    """
    G = np.array([[1, 2], [3, 4]], dtype=np.complex128)
    c = oracle.decompose_full(G)
    np.testing.assert_array_equal(c, np.array([2.5, 2.5, -0.5j, -1.5]))
    g = _rand(1, 7)
    c = oracle.decompose_full(g)
    expect = np.array([(g[0, 0] + g[1, 1]) / 2, (g[0, 1] + g[1, 0]) / 2, 1j * (g[0, 1] - g[1, 0]) / 2,
                       (g[0, 0] - g[1, 1]) / 2])
    np.testing.assert_allclose(c, expect, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_matches_kronecker_trace(N):
    """Eq. (13) (the C oracle) against Tr(P_n G)/2^N with explicit Kronecker tensors (Eq. (4))."""
    G = _rand(N, 100 + N)
    np.testing.assert_allclose(oracle.decompose_full(G), kron.decompose(G), rtol=0, atol=1e-14)


@pytest.mark.parametrize("N", [2, 4])
def test_integer_input_is_exact(N):
    """Integer entries: every partial sum is exact in FP64, so both formulations agree bitwise."""
    G = workloads.integer_complex(N, 5 + N)
    np.testing.assert_array_equal(oracle.decompose_full(G), kron.decompose(G))


def test_one_hot_for_every_pauli_string():
    N = 3
    for n in range(4 ** N):
        c = oracle.decompose_full(kron.pauli_tensor(n, N))
        assert c[n] == 1 and np.count_nonzero(c) == 1


def test_identity():
    c = oracle.decompose_full(np.eye(32, dtype=np.complex128))
    assert c[0] == 1 and np.count_nonzero(c) == 1


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_reconstruction(N):
    """Eq. (1): G = sum_n c_n P_n, with both compose formulations."""
    G = _rand(N, 200 + N)
    c = oracle.decompose_full(G)
    np.testing.assert_allclose(oracle.compose_full(c), G, rtol=0, atol=1e-13)
    np.testing.assert_allclose(kron.compose(c), G, rtol=0, atol=1e-13)


def test_compose_one_hot_is_pauli_tensor():
    N = 2
    for n in range(16):
        e = np.zeros(16, dtype=np.complex128)
        e[n] = 1
        np.testing.assert_array_equal(oracle.compose_full(e), kron.pauli_tensor(n, N))


def test_parseval():
    """The P_n are orthogonal with Tr(P_n^H P_m) = 2^N delta: sum |c|^2 = 2^-N ||G||_F^2."""
    N = 5
    G = _rand(N, 300)
    c = oracle.decompose_full(G)
    assert np.isclose(np.sum(np.abs(c) ** 2), np.linalg.norm(G) ** 2 / 2 ** N, rtol=1e-13)


def test_hermitian_gives_real_coefficients():
    N = 5
    G = workloads.hermitian_complex(N, 301)
    c = oracle.decompose_full(G)
    assert np.max(np.abs(c.imag)) <= 1e-15 * np.max(np.abs(G))


def test_diagonal_input_is_sylvester_hadamard():
    """Diagonal G: only tensors of I and Z survive, and they form 2^-N H diag(G) (scipy's H)."""
    N = 5
    D = 1 << N
    d = _rand(N, 302)[0]
    c = oracle.decompose_full(np.diag(d))
    H = scipy.linalg.hadamard(D)
    expect = (H @ d) / D
    # the tensor whose operator t is Z when bit t of z is set, I otherwise
    n_of_z = [sum(3 << (2 * t) for t in range(N) if (z >> t) & 1) for z in range(D)]
    np.testing.assert_allclose(c[n_of_z], expect, rtol=0, atol=1e-14)
    mask = np.ones(4 ** N, dtype=bool)
    mask[n_of_z] = False
    assert np.count_nonzero(c[mask]) == 0


def test_kronecker_factorisation():
    """decompose(A (x) B)[nA 4^NB + nB] = a[nA] b[nB] (the Pauli basis is a tensor basis)."""
    A, B = _rand(2, 303), _rand(2, 304)
    a, b = oracle.decompose_full(A), oracle.decompose_full(B)
    c = oracle.decompose_full(np.kron(A, B))
    np.testing.assert_allclose(c, np.outer(a, b).ravel(), rtol=0, atol=1e-14)


def test_linearity():
    A, B = _rand(4, 305), _rand(4, 306)
    s = 0.25 - 1.5j
    np.testing.assert_allclose(oracle.decompose_full(A + s * B),
                               oracle.decompose_full(A) + s * oracle.decompose_full(B), rtol=0, atol=1e-14)


def test_sampled_equals_full():
    N = 5
    G = _rand(N, 307)
    full = oracle.decompose_full(G)
    idx = workloads.sample_indices(N, 308, k=200)
    np.testing.assert_array_equal(oracle.decompose_at(G, idx), full[idx.astype(np.int64)])


def _gray_code_coefficient(G, n, N):
    """The paper's fast variant restated (Sec. 3 and Eq. (14)): visit i in Gray-code order and
    update lambda by one factor per step instead of rebuilding it."""
    P = kron.PAULIS
    dig = kron.digits(n, N)
    m = sum(1 << t for t in range(N) if dig[t] in (1, 2))

    def beta(t, i):
        a = (i >> t) & 1
        return P[dig[t]][a, a ^ ((m >> t) & 1)]

    lam = np.prod([beta(t, 0) for t in range(N)]) if N else 1.0
    total = lam * G[m, 0]
    prev = 0
    for k in range(1, 1 << N):
        i = k ^ (k >> 1)
        t = (i ^ prev).bit_length() - 1
        lam = lam * beta(t, i) / beta(t, prev)
        total += lam * G[i ^ m, i]
        prev = i
    return total / (1 << N)


@pytest.mark.parametrize("N", [1, 3, 5])
def test_gray_code_variant_agrees(N):
    G = _rand(N, 309 + N)
    idx = range(4 ** N) if N < 5 else workloads.sample_indices(N, 310, k=64)
    idx = [int(i) for i in idx]
    fast = np.array([_gray_code_coefficient(G, n, N) for n in idx])
    np.testing.assert_allclose(oracle.decompose_at(G, idx), fast, rtol=0, atol=1e-13)


def test_adjoint_dot_product():
    """<decompose(G), y> = <G, 2^-N compose(y)> with <u, v> = sum conj(u) v."""
    N = 3
    G = _rand(N, 311)
    y = workloads.gaussian_complex(3, 312).ravel()  # 64 = 4^3 values
    lhs = np.vdot(oracle.decompose_full(G), y)
    rhs = np.vdot(G.ravel(), oracle.compose_full(y).ravel() * 2.0 ** -N)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gradient_of_weighted_norm_by_finite_differences():
    """loss = sum_n w_n |c_n|^2; torch's grad_c = 2 w c; grad_G = decompose_grad(grad_c)
    should equal dL/dRe(G) + i dL/dIm(G) (central differences)."""
    N = 2
    G = _rand(N, 313)
    w = np.random.default_rng(314).uniform(size=4 ** N)

    def loss(M):
        return float(np.sum(w * np.abs(oracle.decompose_full(M)) ** 2))

    grad = oracle.decompose_grad(2 * w * oracle.decompose_full(G))
    h = 1e-6
    for (r, q) in [(0, 0), (1, 3), (3, 2), (2, 2)]:
        E = np.zeros_like(G)
        E[r, q] = 1
        d_re = (loss(G + h * E) - loss(G - h * E)) / (2 * h)
        d_im = (loss(G + 1j * h * E) - loss(G - 1j * h * E)) / (2 * h)
        assert abs(grad[r, q] - (d_re + 1j * d_im)) < 1e-7


@pytest.mark.parametrize("N", [1, 3])
def test_weighted_norm_unit_weights_is_parseval(N):
    """w = 1: sum_n |c_n|^2 = 2^-N ||G||_F^2, from Tr(P_m P_n) = 2^N [m = n] (Sec. 2)."""
    G = _rand(N, 320 + N)
    want = float(np.sum(np.abs(G) ** 2)) / 2 ** N
    got = oracle.weighted_norm(oracle.decompose_full(G), np.ones(4 ** N))
    assert abs(got - want) <= 1e-13 * want


def test_weighted_norm_one_hot_and_batch():
    N = 2
    w = np.random.default_rng(330).uniform(size=4 ** N)
    for k in (0, 5, 15):
        c = np.zeros(4 ** N, dtype=np.complex128)
        c[k] = 3 - 4j
        assert oracle.weighted_norm(c, w) == 25.0 * w[k]
    cb = workloads.gaussian_complex(N, 331).reshape(1, -1)[:, :16].repeat(3, axis=0) * np.array([[1], [2j], [-3]])
    parts = [oracle.weighted_norm(row, w) for row in cb]
    assert abs(oracle.weighted_norm(cb, w) - sum(parts)) <= 1e-14 * sum(parts)
    assert abs(parts[1] - 4 * parts[0]) <= 1e-14 * parts[1] and abs(parts[2] - 9 * parts[0]) <= 1e-14 * parts[2]


def test_weighted_norm_grad_by_finite_differences():
    """g (dL/dRe c + i dL/dIm c) by central differences against weighted_norm_grad."""
    N = 2
    rng = np.random.default_rng(332)
    c = rng.normal(size=4 ** N) + 1j * rng.normal(size=4 ** N)
    w = rng.uniform(size=4 ** N)
    g = 1.5
    grad = oracle.weighted_norm_grad(c, w, g)
    h = 1e-6
    for k in (0, 7, 15):
        e = np.zeros_like(c)
        e[k] = 1
        d_re = (oracle.weighted_norm(c + h * e, w) - oracle.weighted_norm(c - h * e, w)) / (2 * h)
        d_im = (oracle.weighted_norm(c + 1j * h * e, w) - oracle.weighted_norm(c - 1j * h * e, w)) / (2 * h)
        assert abs(grad[k] - g * (d_re + 1j * d_im)) < 1e-7


@pytest.mark.parametrize("N", [1, 3])
def test_real_part_is_the_hermitian_part(N):
    """Re c_n(G) = c_n((G + G^H)/2): every P_n is Hermitian, so Tr(P_n G^H) = conj Tr(P_n G)
    (the identity the real-part decomposition relies on)."""
    G = _rand(N, 340 + N)
    H = (G + G.conj().T) / 2
    np.testing.assert_allclose(oracle.decompose_full(G).real, oracle.decompose_full(H).real, rtol=0, atol=1e-14)
    assert np.max(np.abs(oracle.decompose_full(H).imag)) <= 1e-14


def test_real_matrix_coefficients():
    """Real G: c_n is real for an even number of Y factors and imaginary for an odd number (each
    Y entry is imaginary, Eq. (3)), exactly in the oracle's sums; iY (real) decomposes to the
    one-hot a_Y = 1, and X (x) iY to the one-hot a at the (X, Y) index."""
    iY = np.array([[0.0, 1.0], [-1.0, 0.0]])
    a = oracle.real_coefficients_at(iY, range(4))
    np.testing.assert_array_equal(a, [0.0, 0.0, 1.0, 0.0])
    X = np.array([[0.0, 1.0], [1.0, 0.0]])
    a2 = oracle.real_coefficients_at(np.kron(X, iY), range(16))
    want = np.zeros(16)
    want[4 * 1 + 2] = 1.0  # operator 1 = X (digit 1), operator 0 = Y (digit 2)
    np.testing.assert_array_equal(a2, want)
    N = 3
    G = np.random.default_rng(350).normal(size=(8, 8))
    c = oracle.decompose_full(G.astype(np.complex128))
    k = oracle.y_count(range(4 ** N), N)
    assert np.all(c.imag[k % 2 == 0] == 0.0) and np.all(c.real[k % 2 == 1] == 0.0)
    a = oracle.real_coefficients_at(G, range(4 ** N))
    np.testing.assert_array_equal(np.where(k % 2 == 1, c.imag, c.real), a)


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.decompose_at(np.zeros((3, 3)), [0])
    with pytest.raises(ValueError):
        oracle.decompose_at(np.zeros((4, 4)), [16])
    with pytest.raises(ValueError):
        oracle.compose_at(np.zeros(15), [0], [0])


# ---- the compensated sum ---------------------------------------------------------------------
# A plain FP64 running sum of 2^N terms can lose every small term next to a large one; the
# oracle's Neumaier sum must not. These pins use integer data whose exact sums Python integers
# (and numpy int64) compute without rounding: a diagonal holding +-2^60 first and last and small
# integers in between. Every partial sum of a plain running sum is then +-2^60 (the small terms
# fall below its 256-wide ulp) and the final result loses all of them, while the compensated sum
# returns the exactly rounded total. The diagonal matrix needs only the x = 0 coefficients
# (Z/I strings), which are a Sylvester-Hadamard transform of the diagonal (scipy.linalg.hadamard)
# divided by 2^N (Eq. (4) with P_n diagonal).

_BIG = 2 ** 60


def _cancelling_diagonal(N, seed):
    """Integer diagonal: +2^60 first, -2^60 last, small integers in [-5, 5] in between."""
    D = 1 << N
    rng = np.random.default_rng(seed)
    d = rng.integers(-5, 6, size=D).astype(np.int64)
    d[0], d[-1] = _BIG, -_BIG
    return d


def _z_string_index(z, N):
    """Tensor index of the string with Z where z has a set bit and I elsewhere (digit 3 = Z)."""
    return sum(3 << (2 * t) for t in range(N) if (z >> t) & 1)


def _exact_hadamard_over_d(d, N):
    """round-to-nearest(H d) * 2^-N with H d in exact int64 arithmetic (|H d| < 2^62)."""
    H = scipy.linalg.hadamard(1 << N, dtype=np.int64)
    s = H @ d
    return np.array([float(int(v)) for v in s]) * 2.0 ** -N  # int -> float rounds correctly


@pytest.mark.parametrize("N", [10, 12])
def test_compensated_sum_is_exact_on_cancelling_diagonal(N):
    """Eq. (13) summed with compensation: bit-exact on sums that a plain FP64 sum gets wrong."""
    D = 1 << N
    dre = _cancelling_diagonal(N, 31 + N)
    dim = _cancelling_diagonal(N, 57 + N)
    dim[0], dim[-1] = -_BIG, _BIG  # the opposite order of signs in the imaginary part
    G = np.zeros((D, D), dtype=np.complex128)
    G[np.arange(D), np.arange(D)] = dre.astype(np.float64) + 1j * dim.astype(np.float64)
    idx = np.array([_z_string_index(z, N) for z in range(D)], dtype=np.uint64)
    got = oracle.decompose_at(G, idx)
    np.testing.assert_array_equal(got.real, _exact_hadamard_over_d(dre, N))
    np.testing.assert_array_equal(got.imag, _exact_hadamard_over_d(dim, N))
    # the identity coefficient is the trace / 2^N: the small terms alone survive the cancellation
    assert got[0].real == float(int(dre[1:-1].sum())) * 2.0 ** -N
    assert got[0].real != 0.0  # what a plain running sum returns


def test_compensated_sum_is_exact_in_composition():
    """Eq. (1) summed with compensation: [G]_{rr} = sum over I/Z strings n of c_n (-1)^popc(r & z(n)),
    i.e. the Sylvester-Hadamard transform of the I/Z coefficients, exact in int64 and rounded once."""
    N = 8
    D = 1 << N
    cz = _cancelling_diagonal(N, 91)  # c of the I/Z string with Z-mask z, for z = 0 .. D-1
    c = np.zeros(4 ** N, dtype=np.complex128)
    for z in range(D):
        c[_z_string_index(z, N)] = float(cz[z])
    # n = 0 (all I) holds +2^60 and n = 4^N - 1 (all Z) holds -2^60: first and last in the sum
    assert c[0] == _BIG and c[4 ** N - 1] == -_BIG
    r = np.arange(D, dtype=np.uint64)
    got = oracle.compose_at(c, r, r)
    H = scipy.linalg.hadamard(D, dtype=np.int64)
    want = np.array([float(int(v)) for v in H @ cz])
    np.testing.assert_array_equal(got.real, want)
    assert np.all(got.imag == 0)
    assert got[0].real == float(int(cz[1:-1].sum())) and got[0].real != 0.0
