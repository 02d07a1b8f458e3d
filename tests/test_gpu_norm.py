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


@pytest.mark.parametrize("fused", [True, False])
def test_adjoint_workload_full_size(fused):
    """64 matrices at N = 10 (the adjoint workload, same calls as the benchmark): the loss
    against the oracle's per-matrix norms of the GPU coefficients, the coefficients and the
    gradient at sampled entries against the oracle."""
    N, B = 10, 64
    A = workloads.adjoint_inputs(workloads.SEEDS["adjoint"], batch=B, N=N)
    w = workloads.adjoint_weights(workloads.SEEDS["adjoint_w"], N)
    Gt = _dev(A).requires_grad_(True)
    if fused:
        loss, c = pg.decompose_weighted_norm_autograd(Gt, _dev(w))
    else:
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


# ----------------------------------------------------------------------------- fused forms --
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,count", [(3, 2), (6, 1), (7, 5), (10, 3), (11, 2), (12, 1), (12, 2)])
def test_decompose_weighted_norm_matches_oracle(N, count, dtype):
    """One fused pass (N 6..12) or decomposition + norm (N < 6): the coefficients equal the plain
    decomposition's (bit for bit in complex128: every single-pass shape computes identical
    values) and the loss the oracle's norm of them."""
    G = np.stack([workloads.gaussian_complex(N, 960 + k) for k in range(count)]).astype(NP[dtype])
    w = workloads.adjoint_weights(961 + N, N).astype(RT[dtype])
    Gd = _dev(G)
    c, loss = pg.decompose_weighted_norm(Gd, _dev(w))
    ch = c.cpu().numpy()
    # the reference decomposition in a single-pass shape (N = 12 defaults to the two-stage kernel)
    op = "decompose_batched" if count > 1 else "decompose"
    if N >= 12:
        pg.set_variant(N, dtype, op, "unit8192")
    try:
        ref = pg.decompose(Gd).cpu().numpy()
    finally:
        if N >= 12:
            pg.set_variant(N, dtype, op, "default")
    if dtype == torch.complex128:
        np.testing.assert_array_equal(ch, ref)
    else:
        assert np.max(np.abs(ch - ref)) <= 2e-6 * np.max(np.abs(G))
    want = oracle.weighted_norm(ch, w)
    assert abs(float(loss.cpu()) - want) <= LOSS_TOL[dtype] * want
    idx = workloads.sample_indices(N, 962, k=128)
    want_c = oracle.decompose_at(G[0].astype(np.complex128), idx)
    tol = {torch.complex128: 1e-12, torch.complex64: 2e-6}[dtype]
    assert np.max(np.abs(ch[0][idx.astype(np.int64)] - want_c)) <= tol * np.max(np.abs(G[0]))


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,count", [(2, 3), (5, 2), (6, 1), (8, 4), (10, 3), (12, 1)])
def test_compose_weighted_matches_grad_then_compose(N, count, dtype):
    """compose_weighted(c, w, g, 1 - N) = compose(weighted_norm_grad(c, w, g), -N): bit for bit
    in complex128; and at sampled entries against the oracle's 2^-N compose(2 g w c)."""
    c = _coeffs(N, count, 970 + N, dtype)
    w = workloads.adjoint_weights(971 + N, N).astype(RT[dtype])
    g = np.array([0.625], dtype=RT[dtype])
    cd, wd, gd = _dev(c), _dev(w), _dev(g)
    got = pg.compose_weighted(cd, wd, gd, scale_exp=1 - N).cpu().numpy()
    two = pg.compose(pg.weighted_norm_grad(cd, wd, gd), scale_exp=-N).cpu().numpy()
    scale = np.max(np.abs(two))
    if dtype == torch.complex128:
        np.testing.assert_array_equal(got, two)
    else:
        assert np.max(np.abs(got - two)) <= 1e-5 * scale
    D = 1 << N
    rows = np.arange(0, D, max(1, D // 64))
    cols = (rows * 5 + 1) % D
    for k in (0, count - 1):
        want = oracle.compose_at(oracle.weighted_norm_grad(c[k], w.astype(np.float64), 0.625), rows, cols) * 2.0 ** -N
        tol = {torch.complex128: 1e-12, torch.complex64: 1e-5}[dtype]
        assert np.max(np.abs(got[k][rows, cols] - want)) <= tol * np.max(np.abs(want)) * max(1, N)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N,count", [(4, 3), (6, 2), (10, 2)])
def test_fused_adjoint_chain_matches_oracle(N, count, dtype):
    """decompose_weighted_norm_autograd: L and dL/dG against the oracle (fused kernels for
    N >= 6; the plain weighted composition below)."""
    G = np.stack([workloads.gaussian_complex(N, 980 + k) for k in range(count)]).astype(NP[dtype])
    w = workloads.adjoint_weights(981, N)
    Gt = _dev(G).requires_grad_(True)
    loss, c = pg.decompose_weighted_norm_autograd(Gt, _dev(w.astype(RT[dtype])))
    assert not c.requires_grad
    (3.0 * loss).backward()
    w_used = w.astype(RT[dtype]).astype(np.float64)
    tol = {torch.complex128: 1e-12, torch.complex64: 1e-5}[dtype]
    if N <= 6:
        c_ref = np.stack([oracle.decompose_full(G[k].astype(np.complex128)) for k in range(count)])
        want_loss = oracle.weighted_norm(c_ref, w_used)
        want = np.stack([oracle.decompose_grad(oracle.weighted_norm_grad(c_ref[k], w_used, 3.0)) for k in range(count)])
        got = Gt.grad.cpu().numpy()
        assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    else:
        ch = c.cpu().numpy()
        want_loss = oracle.weighted_norm(ch, w_used)
        D = 1 << N
        rows = np.arange(0, D, 29)
        cols = (rows * 3 + 7) % D
        got = Gt.grad.cpu().numpy()
        for k in range(count):
            want = oracle.compose_at(oracle.weighted_norm_grad(ch[k], w_used, 3.0), rows, cols) * 2.0 ** -N
            assert np.max(np.abs(got[k][rows, cols] - want)) <= tol * np.max(np.abs(want)) * N
    assert abs(float(loss.detach().cpu()) - want_loss) <= tol * want_loss


def test_fused_adjoint_falls_back_above_n12():
    """N = 13: the forward is the tiled decomposition + the norm, the backward the gradient +
    composition (no fused kernel at this size); checked at sampled entries."""
    N = 13
    G = workloads.gaussian_complex(N, 990)
    w = workloads.adjoint_weights(991, N)
    Gt = _dev(G).requires_grad_(True)
    loss, c = pg.decompose_weighted_norm_autograd(Gt, _dev(w))
    loss.backward()
    ch = c.cpu().numpy()
    want_loss = oracle.weighted_norm(ch, w)
    assert abs(float(loss.detach().cpu()) - want_loss) <= 1e-12 * want_loss
    idx = workloads.sample_indices(N, 992, k=64)
    assert np.max(np.abs(ch[idx.astype(np.int64)] - oracle.decompose_at(G, idx))) <= 1e-12 * np.max(np.abs(G))
    # dL/dG = 2^-N compose(2 w c), so its coefficients are 2^(1-N) w c: decompose sampled
    # coefficients of the GPU gradient with the oracle (O(2^N) each at this size)
    gidx = workloads.sample_indices(N, 993, k=64)
    want = 2.0 ** (1 - N) * w[gidx.astype(np.int64)] * ch[gidx.astype(np.int64)]
    got = oracle.decompose_at(Gt.grad.cpu().numpy(), gidx)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_fused_nonfinite_and_zero_weights():
    """A NaN in G makes its class's coefficients and the loss NaN (as in the separate calls);
    zero weights drop their coefficients from the loss and from the weighted composition."""
    N = 8
    G = workloads.gaussian_complex(N, 995)
    w = workloads.adjoint_weights(996, N)
    Gn = G.copy()
    Gn[3, 17] = np.nan
    c, loss = pg.decompose_weighted_norm(_dev(Gn), _dev(w))
    assert np.isnan(float(loss.cpu()))
    ch = c.cpu().numpy()
    ref = pg.decompose(_dev(Gn)).cpu().numpy()
    np.testing.assert_array_equal(np.isnan(ch), np.isnan(ref))
    wz = w.copy()
    wz[::3] = 0.0
    c, loss = pg.decompose_weighted_norm(_dev(G), _dev(wz))
    ch = c.cpu().numpy()
    want = oracle.weighted_norm(ch, wz)
    assert abs(float(loss.cpu()) - want) <= 1e-12 * want
    cz = ch.copy()
    cz[::3] = 0.0
    a = pg.compose_weighted(_dev(ch), _dev(wz)).cpu().numpy()
    b = pg.compose_weighted(_dev(cz), _dev(wz)).cpu().numpy()
    np.testing.assert_array_equal(a, b)
