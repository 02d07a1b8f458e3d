"""GPU parity of the real-matrix decomposition pauli_decompose_real: against the oracle's
a_n (c_n = i^(k mod 2) a_n, k the number of Y factors), and bit for bit against the nonzero
part that pauli_decompose stores for G + 0i with the same launch shape.

Tolerance as for complex128: 1e-12 max|G|.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import workloads

pytestmark = pytest.mark.gpu


def _real(N, seed, count=None):
    rng = np.random.default_rng(seed)
    shape = (1 << N, 1 << N) if count is None else (count, 1 << N, 1 << N)
    return rng.standard_normal(shape)


def _nonzero_part(c, N):
    k = oracle.y_count(np.arange(4 ** N), N)
    return np.where(k % 2 == 1, c.imag, c.real)


@pytest.mark.parametrize("N", [1, 3, 5, 6, 7, 9, 12, 13, 14])
def test_real_matches_oracle_and_complex_path(N):
    G = _real(N, 1800 + N)
    Gd = torch.from_numpy(G).cuda()
    # both paths follow the complex128 decomposition's launch shape: pin it for the two calls
    if 6 <= N <= 12:
        pg.set_variant(N, torch.complex128, "decompose", "unit8192" if N >= 7 else "unit4096")
    try:
        got = pg.decompose_real(Gd).cpu().numpy()
        full = pg.decompose(Gd.to(torch.complex128), method="auto" if N >= 6 else "plain").cpu().numpy()
    finally:
        if 6 <= N <= 12:
            pg.set_variant(N, torch.complex128, "decompose", "default")
    idx = np.arange(4 ** N, dtype=np.uint64) if N <= 6 else workloads.sample_indices(N, 1810 + N, k=512)
    want = oracle.real_coefficients_at(G, idx)
    assert np.max(np.abs(got[idx.astype(np.int64)] - want)) <= 1e-12 * np.max(np.abs(G)), N
    # the complex path on G + 0i, same launch shape: its nonzero parts, bit for bit
    np.testing.assert_array_equal(got, _nonzero_part(full, N))


def test_real_batch_plain_method_and_errors():
    N, count = 8, 3
    G = _real(N, 1830, count)
    Gd = torch.from_numpy(G).cuda()
    got = pg.decompose_real(Gd).cpu().numpy()
    for k in range(count):
        idx = workloads.sample_indices(N, 1831 + k, k=256)
        want = oracle.real_coefficients_at(G[k], idx)
        assert np.max(np.abs(got[k][idx.astype(np.int64)] - want)) <= 1e-12 * np.max(np.abs(G[k]))
    plain = pg.decompose_real(Gd, method="plain").cpu().numpy()
    assert np.max(np.abs(plain - got)) <= 2e-12 * np.max(np.abs(G))
    with pytest.raises(TypeError):
        pg.decompose_real(Gd.to(torch.float32))
    with pytest.raises(pg.PauliError):
        pg.decompose_real(Gd[0], out=Gd[0].view(-1))
