"""GPU parity of the weighted coefficient norm L = sum_k sum_n w_n |c_{k,n}|^2 and its gradient
2 g w c (pauli_weighted_norm, pauli_weighted_norm_grad) against the oracle, and of the whole
adjoint chain G -> c -> L -> dL/dG through the two autograd Functions.

Tolerances (from the arithmetic): complex128 -- the loss within 1e-12 relative (FP64 terms,
a few thousand sequential additions per thread), the gradient bit for bit (2 g w_n and its
product with c round exactly as the oracle's FP64 expression does); complex64 -- the loss
within 1e-6 relative (three FP32 roundings per term, compensated sums) and the gradient within
1e-6 of its largest element (two FP32 roundings).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import workloads

pytestmark = pytest.mark.gpu

NP = {torch.complex128: np.complex128, torch.complex64: np.complex64}
RT = {torch.complex128: np.float64, torch.complex64: np.float32}
LOSS_TOL = {torch.complex128: 1e-12, torch.complex64: 1e-6}


def _coeffs(N, count, seed, dtype):
    rng = np.random.default_rng(seed)
    c = rng.normal(size=(count, 4 ** N)) + 1j * rng.normal(size=(count, 4 ** N))
    c[:, ::5] *= 1e-3  # a spread of magnitudes
    return c.astype(NP[dtype])


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# (N, count): flat form (count < 4), per-n form with 4^N < 2^18 (several vectors per n
# thread) and 4^N >= 2^18 (several n per thread), ragged batch sizes
SHAPES = [(1, 1), (2, 3), (3, 4), (5, 1), (5, 7), (8, 5), (9, 4), (9, 1), (10, 2), (10, 9)]


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,count", SHAPES)
def test_weighted_norm_matches_oracle(N, count, dtype):
    c = _coeffs(N, count, 900 + 16 * N + count, dtype)
    w = workloads.adjoint_weights(901 + N, N).astype(RT[dtype])
    got = float(pg.weighted_norm(_dev(c), _dev(w)).cpu())
    want = oracle.weighted_norm(c, w)
    assert abs(got - want) <= LOSS_TOL[dtype] * want, (got, want)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,count", [(2, 3), (5, 7), (9, 4), (10, 2)])
def test_weighted_norm_grad_matches_oracle(N, count, dtype):
    c = _coeffs(N, count, 910 + N, dtype)
    w = workloads.adjoint_weights(911 + N, N).astype(RT[dtype])
    g = np.array(0.75, dtype=RT[dtype])
    got = pg.weighted_norm_grad(_dev(c), _dev(w), _dev(g.reshape(1))).cpu().numpy()
    if dtype == torch.complex128:
        np.testing.assert_array_equal(got, oracle.weighted_norm_grad(c, w, 0.75))
        np.testing.assert_array_equal(pg.weighted_norm_grad(_dev(c), _dev(w)).cpu().numpy(),
                                      oracle.weighted_norm_grad(c, w))
    else:
        want = oracle.weighted_norm_grad(c, w, 0.75)
        assert np.max(np.abs(got - want)) <= 1e-6 * np.max(np.abs(want))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_weighted_norm_deterministic_and_in_place_grad(dtype):
    N, count = 9, 6
    c = _dev(_coeffs(N, count, 920, dtype))
    w = _dev(workloads.adjoint_weights(921, N).astype(RT[dtype]))
    a = pg.weighted_norm(c, w).cpu()
    b = pg.weighted_norm(c, w).cpu()
    assert a.numpy().tobytes() == b.numpy().tobytes()
    sep = pg.weighted_norm_grad(c, w)
    pg.weighted_norm_grad(c, w, out=c)
    torch.cuda.synchronize()
    assert torch.equal(sep, c)


def test_weighted_norm_rejects_aliasing_and_bad_weights():
    c = _dev(_coeffs(3, 2, 930, torch.complex128))
    w = _dev(np.ones(64))
    with pytest.raises(pg.PauliError):
        pg.weighted_norm(c, w, out=c.view(torch.float64).view(-1)[0])
    with pytest.raises(ValueError):
        pg.weighted_norm(c, _dev(np.ones(63)))
    with pytest.raises(ValueError):
        pg.weighted_norm(c, _dev(np.ones(64, dtype=np.float32)))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,count", [(4, 3), (6, 5)])
def test_adjoint_chain_matches_oracle(N, count, dtype):
    """L(G) = sum_k sum_n w_n |c_n(G_k)|^2 and dL/dG through decompose_autograd and
    weighted_norm_autograd (kernels only) against the oracle's decompose, norm and
    2^-N compose(2 w c)."""
    G = np.stack([workloads.gaussian_complex(N, 940 + k) for k in range(count)]).astype(NP[dtype])
    w = workloads.adjoint_weights(941, N)
    Gt = _dev(G).requires_grad_(True)
    loss = pg.weighted_norm_autograd(pg.decompose_autograd(Gt), _dev(w.astype(RT[dtype])))
    loss.backward()
    c_ref = np.stack([oracle.decompose_full(G[k]) for k in range(count)])
    w_used = w.astype(RT[dtype]).astype(np.float64)
    want_loss = oracle.weighted_norm(c_ref, w_used)
    tol = {torch.complex128: 1e-12, torch.complex64: 1e-5}[dtype]
    assert abs(float(loss.detach().cpu()) - want_loss) <= tol * want_loss
    want = np.stack([oracle.decompose_grad(oracle.weighted_norm_grad(c_ref[k], w_used)) for k in range(count)])
    got = Gt.grad.cpu().numpy()
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


def test_adjoint_workload_full_size():
    """64 matrices at N = 10 (the adjoint workload, same calls as the benchmark): the loss
    against the oracle's per-matrix norms of the GPU coefficients, the coefficients and the
    gradient at sampled entries against the oracle."""
    N, B = 10, 64
    A = workloads.adjoint_inputs(workloads.SEEDS["adjoint"], batch=B, N=N)
    w = workloads.adjoint_weights(workloads.SEEDS["adjoint_w"], N)
    Gt = _dev(A).requires_grad_(True)
    c = pg.decompose_autograd(Gt)
    loss = pg.weighted_norm_autograd(c, _dev(w))
    loss.backward()
    ch = c.detach().cpu().numpy()
    want_loss = sum(oracle.weighted_norm(ch[k], w) for k in range(B))
    assert abs(float(loss.detach().cpu()) - want_loss) <= 1e-12 * want_loss
    for k in (0, 37, 63):
        idx = workloads.sample_indices(N, 950 + k, k=64)
        ref = oracle.decompose_at(A[k], idx)
        assert np.max(np.abs(ch[k][idx.astype(np.int64)] - ref)) <= 1e-12 * np.max(np.abs(A[k]))
    D = 1 << N
    rows = np.arange(0, D, 61)
    cols = (rows * 7 + 11) % D
    gh = Gt.grad.cpu().numpy()
    for k in (0, 63):
        want = oracle.compose_at(oracle.weighted_norm_grad(ch[k], w), rows, cols) * 2.0 ** -N
        assert np.max(np.abs(gh[k][rows, cols] - want)) <= 1e-12 * np.max(np.abs(want)) * 4
