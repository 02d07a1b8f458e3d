"""GPU parity of the real-part (Hermitian) decomposition pauli_decompose_hermitian: against the
oracle's Re c_n, and bit for bit against the real parts pauli_decompose stores with the same
launch shape (the two share every kernel step but the final store).

Tolerances as for the complex decomposition: 1e-12 max|G| (complex128), 2e-6 max|G| (complex64).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import workloads

pytestmark = pytest.mark.gpu

NP = {torch.complex128: np.complex128, torch.complex64: np.complex64}
TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _same_shape_variant(N):
    """The launch shape the real-part path takes below N = 13."""
    return "unit8192" if N >= 7 else "unit4096"


def _check_against_oracle(G, got, N, dtype, k=None):
    Gr = G.astype(NP[dtype]).astype(np.complex128)
    if k is None:
        idx = np.arange(4 ** N, dtype=np.uint64)
    else:
        idx = workloads.sample_indices(N, 1700 + N, k=k)
    want = oracle.decompose_at(Gr, idx).real
    err = np.max(np.abs(got[idx.astype(np.int64)].astype(np.float64) - want))
    assert err <= TOL[dtype] * np.max(np.abs(Gr)), (N, dtype, err)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,variant", [(1, None), (3, None), (5, None), (6, "same"), (8, "same"), (10, "same"),
                                       (12, "same"), (12, "twostage")])
def test_hermitian_matches_oracle_and_complex_path(N, variant, dtype):
    """Real parts against the oracle, and bit for bit against the real part of the complex
    decomposition in the same launch shape (both calls follow the decomposition's shape)."""
    G = workloads.hermitian_complex(N, 1600 + N).astype(NP[dtype])
    Gd = _dev(G)
    if variant:
        pg.set_variant(N, dtype, "decompose", _same_shape_variant(N) if variant == "same" else variant)
    try:
        got = pg.decompose_hermitian(Gd).cpu().numpy()
        full = pg.decompose(Gd).cpu().numpy()
    finally:
        if variant:
            pg.set_variant(N, dtype, "decompose", "default")
    assert got.dtype == (np.float64 if dtype == torch.complex128 else np.float32)
    _check_against_oracle(G, got, N, dtype, k=None if N <= 8 else 2048)
    np.testing.assert_array_equal(got, full.real)
    # Hermitian input: the dropped imaginary parts are rounding noise
    assert np.max(np.abs(full.imag)) <= TOL[dtype] * np.max(np.abs(G))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N", [13, 14])
def test_hermitian_tiled_matches_oracle_and_complex_path(N, dtype):
    """N = 13, 14: the tiled kernel (the decomposition's built-in shape there); sampled
    oracle check and bitwise equality with the complex path's real parts."""
    G = workloads.hermitian_complex(N, 1600 + N).astype(NP[dtype])
    Gd = _dev(G)
    got = pg.decompose_hermitian(Gd)
    full = pg.decompose(Gd)
    torch.cuda.synchronize()
    assert torch.equal(got, full.real)
    del full
    _check_against_oracle(G, got.cpu().numpy(), N, dtype, k=512)


def test_hermitian_of_general_matrix_is_hermitian_part():
    N = 9
    G = workloads.gaussian_complex(N, 1620)
    H = (G + G.conj().T) / 2
    a = pg.decompose_hermitian(_dev(G)).cpu().numpy()
    b = pg.decompose_hermitian(_dev(H)).cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(G))
    _check_against_oracle(G, a, N, torch.complex128, k=1024)


@pytest.mark.parametrize("N,count", [(4, 5), (7, 3), (12, 2)])
def test_hermitian_batch_and_plain_method(N, count):
    G = np.stack([workloads.hermitian_complex(N, 1630 + k) for k in range(count)])
    Gd = _dev(G)
    got = pg.decompose_hermitian(Gd).cpu().numpy()
    assert got.shape == (count, 4 ** N)
    for k in (0, count - 1):
        _check_against_oracle(G[k], got[k], N, torch.complex128, k=None if N <= 7 else 1024)
    if N <= 7:
        plain = pg.decompose_hermitian(Gd, method="plain").cpu().numpy()
        np.testing.assert_array_equal(plain, pg.decompose(Gd, method="plain").cpu().numpy().real)


def test_hermitian_rejects_bad_output():
    G = _dev(workloads.hermitian_complex(4, 1640))
    with pytest.raises(ValueError):
        pg.decompose_hermitian(G, out=torch.empty(256, dtype=torch.float32, device="cuda"))
    with pytest.raises(pg.PauliError):
        pg.decompose_hermitian(G, out=G.view(torch.float64).view(-1)[:256])


# ------------------------------------------------------ Hermitian G from its upper triangle --
def _from_upper(G):
    """The Hermitian matrix with G's strict upper triangle and the real parts of its diagonal."""
    U = np.triu(G, 1)
    return U + U.conj().T + np.diag(np.diag(G).real)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N", [1, 3, 5, 6, 7, 8, 10, 12])
def test_upper_matches_oracle_and_full_read(N, dtype):
    G = workloads.hermitian_complex(N, 1700 + N).astype(NP[dtype])
    Gd = _dev(G)
    got = pg.decompose_hermitian(Gd, upper=True).cpu().numpy()
    _check_against_oracle(G, got, N, dtype, k=None if N <= 8 else 2048)
    full = pg.decompose_hermitian(Gd).cpu().numpy()
    assert np.max(np.abs(got.astype(np.float64) - full)) <= TOL[dtype] * np.max(np.abs(G))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N", [4, 7, 9, 12])
def test_upper_never_reads_the_lower_triangle(N, dtype):
    """NaN below the diagonal and in the diagonal's imaginary parts change nothing: the result
    is bit for bit that of the Hermitian matrix."""
    G = workloads.hermitian_complex(N, 1720 + N).astype(NP[dtype])
    bad = G.copy()
    low = np.tril_indices(1 << N, -1)
    bad[low] = np.nan
    d = np.diag_indices(1 << N)
    bad.imag[d] = np.where(np.arange(1 << N) % 2 == 0, np.nan, 7.0)
    assert np.all(np.isfinite(bad.real[d]))
    a = pg.decompose_hermitian(_dev(G), upper=True).cpu().numpy()
    b = pg.decompose_hermitian(_dev(bad), upper=True).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    assert np.all(np.isfinite(b))


def test_upper_of_general_matrix_and_batch_and_plain():
    """A non-Hermitian G gives the coefficients of the Hermitian matrix made from its upper
    triangle; batches; the plain method with mirrored reads agrees."""
    N, count = 9, 3
    G = np.stack([workloads.gaussian_complex(N, 1740 + k) for k in range(count)])
    Gd = _dev(G)
    got = pg.decompose_hermitian(Gd, upper=True).cpu().numpy()
    for k in range(count):
        _check_against_oracle(_from_upper(G[k]), got[k], N, torch.complex128, k=1024)
    plain = pg.decompose_hermitian(Gd[:1], upper=True, method="plain").cpu().numpy()
    assert np.max(np.abs(plain[0] - got[0])) <= 1e-12 * np.max(np.abs(G[0]))


def test_upper_rejects_unsupported_sizes():
    G6 = _dev(workloads.hermitian_complex(6, 1750))
    with pytest.raises(pg.PauliError):
        pg.decompose_hermitian(G6, upper=True, method="xordiag")
    # the two-stage upper-triangle mode wants 16-byte aligned matrices: a complex64 view at an odd
    # element offset is refused
    buf = torch.zeros((1 << 26) + 1, dtype=torch.complex64, device="cuda")
    G13 = buf[1:].view(1 << 13, 1 << 13)
    with pytest.raises(pg.PauliError):
        pg.decompose_hermitian(G13, upper=True)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N", [13, 14])
def test_upper_triangle_two_stage_ignores_the_lower_triangle(N, dtype):
    """N = 13, 14: the two-stage kernel in its upper-triangle mode. With the strict lower triangle
    set to NaN and garbage on the diagonal's imaginary parts it gives, bit for bit, the real
    parts that the full-read Hermitian path gives for the intact matrix; and it matches the
    oracle on samples."""
    G = workloads.hermitian_complex(N, 1700 + N).astype(NP[dtype])  # exactly Hermitian
    Gd = _dev(G)
    full = pg.decompose_hermitian(Gd).cpu().numpy()
    del Gd
    D = 1 << N
    bad = G.copy()
    for r in range(D):
        bad[r, :r] = np.nan
    bad[np.arange(D), np.arange(D)] += np.asarray(7j, dtype=NP[dtype])
    up = pg.decompose_hermitian(_dev(bad), upper=True).cpu().numpy()
    del bad
    np.testing.assert_array_equal(up, full)
    if N == 13:
        _check_against_oracle(G, up, N, dtype, k=512)
