"""GPU: pauli_compose_batched -- the inverse map G = sum_n c_n P_n (Eq. (1)) for a batch of
coefficient vectors of uneven N in one launch -- against the CPU oracle's composition on sampled
matrix elements, against the one-matrix composition (the same exact integer transform for
complex128 from N = 6), with the adjoint scale, over more than one table of 1024 matrices, and
captured in a CUDA graph. Tolerances relative to the output's scale: 1e-12 (complex128) and 2e-6
(complex64) times twice the larger of max|c| and the largest sampled |G| element; the oracle
composes the exactly upcast input in FP64."""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}
NP = {torch.complex128: np.complex128, torch.complex64: np.complex64}


def _coeffs(Ns, seed, dtype):
    return [workloads.gaussian_coefficients(int(N), seed * 100003 + b, NP[dtype]) for b, N in enumerate(Ns)]


def _check(cs, outs, dtype, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    for c, o in zip(cs, outs):
        N = (c.size.bit_length() - 1) // 2
        D = 1 << N
        got = o.cpu().numpy()
        cu = c.astype(np.complex128)
        k = D * D if N <= 3 else (24 if N <= 8 else 6)
        flat = np.arange(D * D) if N <= 3 else rng.integers(0, D * D, k)
        r, q = np.divmod(flat, D)
        want = oracle.compose_at(cu, r.astype(np.uint64), q.astype(np.uint64)) * scale
        err = np.max(np.abs(got[r, q] - want))
        ref = max(np.max(np.abs(cu)) * scale, np.max(np.abs(want)))
        assert err <= TOL[dtype] * ref * 2, (N, err, ref)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_compose_batched_config_against_oracle(dtype):
    """The batched workload's N draw (512 matrices, N 3..10) with seeded coefficient vectors."""
    _, Ns = workloads.batched_hermitian(workloads.SEEDS["batched"], batch=512)
    cs = _coeffs(Ns, 77, dtype)
    cd = [torch.from_numpy(c).cuda() for c in cs]
    outs = [torch.full((1 << int(N), 1 << int(N)), float("nan"), dtype=dtype, device="cuda") for N in Ns]
    pg.compose_batched(cd, outs)
    torch.cuda.synchronize()
    _check(cs, outs, dtype, 5)
    if dtype == torch.complex128:  # one composition per matrix: the same integer transform from N = 6
        for c, o, N in zip(cd, outs, Ns):
            if N >= 6:
                assert torch.equal(pg.compose(c), o)


def test_compose_batched_adjoint_scale_and_small_n():
    """scale_exp = -N gives 2^-N sum_n c_n P_n (the adjoint of the decomposition); N = 1..5 are
    composed whole, exactly (power-of-two scale)."""
    Ns = [1, 2, 3, 4, 5, 6, 7]
    for N in Ns:
        cs = _coeffs([N] * 3, 300 + N, torch.complex128)
        cd = [torch.from_numpy(c).cuda() for c in cs]
        a = pg.compose_batched(cd, scale_exp=-N)
        b = pg.compose_batched(cd)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x, y * 2.0 ** -N)
        _check(cs, b, torch.complex128, 600 + N)


def test_compose_batched_more_than_one_table():
    """1500 matrices: two launches (1024 + 476), every output written."""
    rng = np.random.default_rng(31)
    Ns = rng.integers(1, 5, size=1500)
    cs = _coeffs(Ns, 31, torch.complex128)
    cd = [torch.from_numpy(c).cuda() for c in cs]
    outs = [torch.full((1 << int(N), 1 << int(N)), float("nan"), dtype=torch.complex128, device="cuda") for N in Ns]
    pg.compose_batched(cd, outs)
    torch.cuda.synchronize()
    assert not any(torch.isnan(o).any().item() for o in outs)
    pick = rng.choice(1500, 40, replace=False)
    _check([cs[i] for i in pick], [outs[i] for i in pick], torch.complex128, 32)


def test_compose_batched_graph_capture():
    """A captured call replays with its own table (kernel parameters are copied at capture)."""
    Ns = [3, 6, 8, 10, 4]
    cs = _coeffs(Ns, 41, torch.complex128)
    cd = [torch.from_numpy(c).cuda() for c in cs]
    outs = [torch.full((1 << N, 1 << N), float("nan"), dtype=torch.complex128, device="cuda") for N in Ns]
    pg.compose_batched(cd, [torch.empty_like(o) for o in outs])  # warm-up outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        pg.compose_batched(cd, outs)
    assert all(torch.isnan(o).all().item() for o in outs)
    graph.replay()
    torch.cuda.synchronize()
    _check(cs, outs, torch.complex128, 42)
