"""GPU: the x-class shards -- pauli_xhi_layout + pauli_decompose_xhi for every x_hi of a
matrix, against the CPU oracle (all coefficients for small N, seeded samples per shard above),
with the one-pass (k <= 4) and the multi-pass (k > 4) combine, and the union of the shards
against the one-matrix decomposition. Tolerances relative to max|G|: 1e-12 (complex128) and
2e-6 (complex64, against the oracle on the exactly upcast input)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import shard, workloads

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}
NP = {torch.complex128: np.complex128, torch.complex64: np.complex64}


def _shards(G, N, k, method="auto"):
    L = torch.empty((1 << N, 1 << (N - k)), dtype=G.dtype, device=G.device)
    outs = []
    for g in range(1 << k):
        pg.xhi_layout(G, k, g, out=L)
        outs.append(pg.decompose_xhi(L, N, k, g, method=method).cpu().numpy())
    torch.cuda.synchronize()
    return outs


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,k", [(2, 1), (5, 2), (7, 3), (8, 4), (8, 5), (9, 7), (10, 1)])
def test_shards_match_the_oracle_everywhere(N, k, dtype):
    G_h = workloads.gaussian_complex(N, 300 + 10 * N + k, NP[dtype])
    want = oracle.decompose_full(G_h.astype(np.complex128))
    outs = _shards(torch.from_numpy(G_h).cuda(), N, k)
    got = shard.assemble(outs, N, k).astype(np.complex128)
    err = np.max(np.abs(got - want)) / np.max(np.abs(G_h))
    assert err <= TOL[dtype], err


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,k", [(12, 2), (13, 3), (14, 1)])
def test_shards_at_large_n_on_samples(N, k, dtype):
    """Each shard on 512 seeded entries (and its first and last), against the oracle."""
    G_h = workloads.gaussian_complex(N, 400 + N, NP[dtype])
    G = torch.from_numpy(G_h).cuda()
    Gu = G_h.astype(np.complex128) if dtype == torch.complex64 else G_h
    rng = np.random.default_rng(N * 7 + k)
    L = torch.empty((1 << N, 1 << (N - k)), dtype=dtype, device="cuda")
    o = torch.empty(L.numel(), dtype=dtype, device="cuda")
    for g in range(1 << k):
        pg.xhi_layout(G, k, g, out=L)
        pg.decompose_xhi(L, N, k, g, out=o)
        j = np.concatenate([[0, o.numel() - 1], rng.integers(0, o.numel(), 512)])
        got = o.cpu().numpy()[j].astype(np.complex128)
        n = shard.shard_indices(N, k, g)[j]
        want = oracle.decompose_at(Gu, n)
        err = np.max(np.abs(got - want)) / np.max(np.abs(G_h))
        assert err <= TOL[dtype], (g, err)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_union_of_shards_matches_the_one_matrix_decomposition(dtype):
    N, k = 11, 2
    G_h = workloads.gaussian_complex(N, 511, NP[dtype])
    G = torch.from_numpy(G_h).cuda()
    full = pg.decompose(G).cpu().numpy()
    got = shard.assemble(_shards(G, N, k), N, k)
    # both round each coefficient from near-exact sums: a few units in the last place apart
    assert np.max(np.abs(got - full)) <= TOL[dtype] * np.max(np.abs(G_h))


def test_plain_method_and_layout_copy():
    """The block-XOR copy is the definition's gather, bit for bit; method PLAIN decomposes the
    blocks with the per-coefficient kernel."""
    N, k = 7, 2
    G_h = workloads.gaussian_complex(N, 71)
    G = torch.from_numpy(G_h).cuda()
    m, M = N - k, 1 << (N - k)
    for g in range(1 << k):
        L = pg.xhi_layout(G, k, g).cpu().numpy()
        for r in range(1 << N):
            cb = (r >> m) ^ g
            assert np.array_equal(L[r], G_h[r, cb * M:(cb + 1) * M])
    want = oracle.decompose_full(G_h)
    got = shard.assemble(_shards(G, N, k, method="plain"), N, k)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(G_h))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_layout_copy_of_unaligned_views(dtype):
    """Buffers at an odd element offset (8-byte aligned complex64) take the element-wise copy."""
    N, k = 6, 3
    D, M = 1 << N, 1 << (N - k)
    G_h = workloads.gaussian_complex(N, 72, NP[dtype])
    gbuf = torch.zeros(D * D + 1, dtype=dtype, device="cuda")
    gbuf[1:] = torch.from_numpy(G_h.reshape(-1)).cuda()
    G = gbuf[1:].view(D, D)
    lbuf = torch.zeros(D * M + 1, dtype=dtype, device="cuda")
    for g in range(1 << k):
        pg.xhi_layout(G, k, g, out=lbuf[1:].view(D, M))
        L = lbuf[1:].view(D, M).cpu().numpy()
        for r in range(D):
            cb = (r >> (N - k)) ^ g
            assert np.array_equal(L[r], G_h[r, cb * M:(cb + 1) * M])


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,k", [(12, 1), (13, 2), (14, 3), (12, 6)])
def test_two_stage_shard_equals_the_full_decomposition(N, k, dtype):
    """N = 12..14 with N - k >= 6: one two-stage launch per shard, reading the layout's tiles and
    writing the compact order -- the same classes, tiles and scales as the full decomposition, so
    the same bits (complex64 too: the same compensated grids)."""
    G_h = workloads.gaussian_complex(N, 700 + N + k, NP[dtype])
    G = torch.from_numpy(G_h).cuda()
    pg.set_variant(N, dtype, "decompose", "twostage")
    try:
        full = pg.decompose(G).cpu().numpy()
    finally:
        pg.set_variant(N, dtype, "decompose", "default")
    L = torch.empty((1 << N, 1 << (N - k)), dtype=dtype, device="cuda")
    for g in (0, (1 << k) - 1, (1 << k) // 3):
        pg.xhi_layout(G, k, g, out=L)
        o = pg.decompose_xhi(L, N, k, g).cpu().numpy()
        np.testing.assert_array_equal(o, full[shard.shard_indices(N, k, g).astype(np.int64)])
