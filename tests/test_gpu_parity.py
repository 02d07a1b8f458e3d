"""GPU parity: libpauli (through the C ABI binding) against the CPU oracle.

Tolerances: max |c - c_oracle| <= 1e-12 max|G| for complex128 and <= 2e-6 max|G| for
complex64, max|G| being the largest complex modulus of the input. Integer-valued inputs
must match bit for bit in complex128 (every partial sum is exact on both sides).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}
NP = {torch.complex128: np.complex128, torch.complex64: np.complex64}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def maxabs(G):
    return float(np.max(np.abs(G)))


def gpu_decompose(G, dtype, method):
    return host(pg.decompose(dev(G.astype(NP[dtype])), method=method))


def ref_for(G, dtype):
    """The oracle sees exactly the values the GPU sees (complex64 inputs upcast exactly)."""
    return G.astype(NP[dtype]).astype(np.complex128)


def assert_close(got, want, G, dtype):
    err = np.max(np.abs(got.astype(np.complex128) - want))
    assert err <= TOL[dtype] * maxabs(G), f"err {err:.3e} > {TOL[dtype]:.0e} * {maxabs(G):.3f}"


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("method", ["plain", "xordiag"])
@pytest.mark.parametrize("N", [1, 2, 3, 5, 7, 8])
def test_full_decomposition_small(N, method, dtype):
    if method == "xordiag" and N < 7:
        pytest.skip("no XOR-diagonal kernel below N=7")
    G = workloads.gaussian_complex(N, 40 + N)
    got = gpu_decompose(G, dtype, method)
    assert_close(got, oracle.decompose_full(ref_for(G, dtype)), G, dtype)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_n6_config_plain(dtype):
    G = workloads.gaussian_complex(6, workloads.SEEDS["n6"])
    got = gpu_decompose(G, dtype, "plain")
    assert_close(got, oracle.decompose_full(ref_for(G, dtype)), G, dtype)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N", [9, 10, 11])
def test_sampled_mid_sizes(N, dtype):
    G = workloads.gaussian_complex(N, 60 + N)
    idx = workloads.sample_indices(N, 70 + N, k=512)
    want = oracle.decompose_at(ref_for(G, dtype), idx)
    for method in ("xordiag", "plain"):
        got = gpu_decompose(G, dtype, method)
        assert_close(got[idx.astype(np.int64)], want, G, dtype)


@pytest.mark.parametrize("which", ["general", "hermitian"])
def test_n12_config_both_methods(which):
    N = 12
    G = (workloads.gaussian_complex(N, workloads.SEEDS["n12"]) if which == "general"
         else workloads.hermitian_complex(N, workloads.SEEDS["n12_herm"]))
    Gd = dev(G)
    cx = pg.decompose(Gd, method="xordiag")
    cp = pg.decompose(Gd, method="plain")
    idx = workloads.sample_indices(N, workloads.SEEDS["n12_idx"])
    want = oracle.decompose_at(G, idx)
    cx, cp = host(cx), host(cp)
    i64 = idx.astype(np.int64)
    assert_close(cx[i64], want, G, torch.complex128)
    assert_close(cp[i64], want, G, torch.complex128)
    # the two GPU methods agree on every coefficient
    assert np.max(np.abs(cx - cp)) <= 2e-12 * maxabs(G)
    if which == "hermitian":
        assert np.max(np.abs(cx.imag)) <= 1e-12 * maxabs(G)
        # the real-part and upper-triangle forms the bench times on the same input
        re = host(pg.decompose_hermitian(Gd))
        up = host(pg.decompose_hermitian(Gd, upper=True))
        assert_close(re[i64], want.real, G, torch.complex128)
        assert_close(up[i64], want.real, G, torch.complex128)
        np.testing.assert_array_equal(re, cx.real)
        assert np.max(np.abs(up - cx.real)) <= 2e-12 * maxabs(G)


@pytest.mark.parametrize("method", ["plain", "xordiag"])
@pytest.mark.parametrize("N", [4, 8, 10])
def test_integer_input_bit_exact(N, method):
    if method == "xordiag" and N < 7:
        pytest.skip("no XOR-diagonal kernel below N=7")
    G = workloads.integer_complex(N, 80 + N)
    got = gpu_decompose(G, torch.complex128, method)
    if N <= 8:
        want = oracle.decompose_full(G)
        np.testing.assert_array_equal(got, want)
    else:
        idx = workloads.sample_indices(N, 90, k=1024)
        np.testing.assert_array_equal(got[idx.astype(np.int64)], oracle.decompose_at(G, idx))


@pytest.mark.parametrize("N", [3, 7])
def test_pauli_tensor_is_one_hot(N):
    from oracle import kron
    rng = np.random.default_rng(N)
    for n in rng.integers(0, 4 ** N, size=6):
        got = gpu_decompose(kron.pauli_tensor(int(n), N), torch.complex128, "auto")
        want = np.zeros(4 ** N)
        want[n] = 1
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N", [2, 5, 7, 10])
def test_compose_matches_oracle_and_reconstructs(N, dtype):
    G = workloads.gaussian_complex(N, 100 + N)
    Gd = dev(G.astype(NP[dtype]))
    cd = pg.decompose(Gd)
    back = host(pg.compose(cd))
    assert np.max(np.abs(back - G.astype(NP[dtype]))) <= 4 * TOL[dtype] * maxabs(G)
    cr = np.random.default_rng(N).standard_normal(4 ** N) + 1j * np.random.default_rng(N + 1).standard_normal(4 ** N)
    got = host(pg.compose(dev(cr.astype(NP[dtype]))))
    D = 1 << N
    rows = np.random.default_rng(7).integers(0, D, 64)
    cols = np.random.default_rng(8).integers(0, D, 64)
    want = oracle.compose_at(cr.astype(NP[dtype]).astype(np.complex128), rows, cols)
    err = np.max(np.abs(got[rows, cols] - want))
    assert err <= TOL[dtype] * np.max(np.abs(cr)) * D


@pytest.mark.parametrize("N", [4, 8])
def test_compose_scale_exp(N):
    cr = workloads.gaussian_complex(N, 5).ravel()
    a = host(pg.compose(dev(cr)))
    b = host(pg.compose(dev(cr), scale_exp=-N))
    np.testing.assert_array_equal(b, a * 2.0 ** -N)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_coeffs_at(dtype):
    N = 9
    G = workloads.gaussian_complex(N, 11)
    idx = workloads.sample_indices(N, 12, k=300)
    got = host(pg.coeffs_at(dev(G.astype(NP[dtype])), torch.from_numpy(idx.astype(np.int64)).cuda()))
    assert_close(got, oracle.decompose_at(ref_for(G, dtype), idx), G, dtype)


def test_coeffs_at_out_of_range_is_nan():
    G = workloads.gaussian_complex(3, 1)
    got = host(pg.coeffs_at(dev(G), torch.tensor([0, 64, 3], dtype=torch.int64).cuda()))
    assert np.isnan(got[1]) and not np.isnan(got[0]) and not np.isnan(got[2])


def test_batched_contiguous_matches_single():
    N, B = 8, 5
    Gs = np.stack([workloads.gaussian_complex(N, 200 + b) for b in range(B)])
    out = host(pg.decompose(dev(Gs)))
    for b in range(B):
        np.testing.assert_array_equal(out[b], gpu_decompose(Gs[b], torch.complex128, "auto"))


def test_list_and_plan_match_oracle():
    Ns = [3, 7, 5, 8, 1]
    Gs = [workloads.hermitian_complex(n, 300 + i) for i, n in enumerate(Ns)]
    Gd = [dev(G) for G in Gs]
    outs = pg.decompose_list(Gd)
    plan = pg.PauliPlan(Ns)
    pouts = [torch.empty(4 ** n, dtype=torch.complex128, device="cuda") for n in Ns]
    plan.bind(Gd, pouts)
    plan.execute()
    assert plan.status() == 0
    for G, o, p in zip(Gs, outs, pouts):
        want = oracle.decompose_full(G)
        assert_close(host(o), want, G, torch.complex128)
        assert_close(host(p), want, G, torch.complex128)


def test_host_round_trip():
    N = 9
    G = workloads.gaussian_complex(N, 400)
    Gh = torch.from_numpy(G).pin_memory()
    oh = torch.empty(4 ** N, dtype=torch.complex128).pin_memory()
    Gd = torch.empty((1 << N, 1 << N), dtype=torch.complex128, device="cuda")
    od = torch.empty(4 ** N, dtype=torch.complex128, device="cuda")
    pg.pauli_decompose_host(Gh, oh, Gd, od)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(oh.numpy(), host(pg.decompose(dev(G))))


def test_adjoint_dot_product_identity():
    N = 7
    G = workloads.gaussian_complex(N, 500)
    y = workloads.gaussian_complex(N, 501).ravel()
    lhs = np.vdot(host(pg.decompose(dev(G))), y)
    rhs = np.vdot(G.ravel(), host(pg.compose(dev(y), scale_exp=-N)).ravel())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_gradcheck_n4():
    G = torch.from_numpy(workloads.gaussian_complex(4, workloads.SEEDS["gradcheck"])).cuda().requires_grad_(True)
    assert torch.autograd.gradcheck(lambda g: pg.decompose_autograd(g), (G,), eps=1e-6, atol=1e-8)


@pytest.mark.parametrize("N", [4, 8])
def test_weighted_norm_gradient_matches_oracle(N):
    G = workloads.gaussian_complex(N, 600 + N)
    w = workloads.adjoint_weights(601, N)
    Gt = dev(G).requires_grad_(True)
    c = pg.decompose_autograd(Gt)
    loss = (torch.from_numpy(w).cuda() * c.abs() ** 2).sum()
    loss.backward()
    c_ref = oracle.decompose_full(G) if N <= 4 else host(c.detach())
    want = oracle.decompose_grad(2 * w * c_ref) if N <= 4 else None
    got = host(Gt.grad)
    if want is not None:
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    else:
        D = 1 << N
        rows = np.arange(0, D, 37)
        cols = (rows * 5 + 3) % D
        want_s = oracle.compose_at(2 * w * c_ref, rows, cols) * 2.0 ** -N
        assert np.max(np.abs(got[rows, cols] - want_s)) <= 1e-12 * np.max(np.abs(want_s)) * D


def test_nonfinite_input_gives_nan():
    N = 8
    G = workloads.gaussian_complex(N, 700)
    G[5, 9] = np.inf
    got = gpu_decompose(G, torch.complex128, "xordiag")
    x = 5 ^ 9
    # every coefficient whose XY-mask is 5 ^ 9 depends on the entry: all NaN
    n_all = np.arange(4 ** N)
    even = sum(((n_all >> (2 * t)) & 1) << t for t in range(N))
    odd = sum(((n_all >> (2 * t + 1)) & 1) << t for t in range(N))
    mask = (even ^ odd) == x
    assert np.all(np.isnan(got[mask]))
    assert not np.any(np.isnan(got[~mask]))


def test_device_errors_with_real_buffers():
    G = dev(workloads.gaussian_complex(8, 1))
    with pytest.raises(pg.PauliError, match="ALIAS"):
        pg.decompose(G, out=G.view(-1))
    with pytest.raises(ValueError):
        pg.decompose(G.cpu())


# ---------------------------------------------------------------- cluster sizes (N >= 13) --
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_n14_config_sampled(dtype):
    """The benchmark workload at full size: 4096 seeded sampled coefficients + special ones."""
    N = 14
    G = workloads.gaussian_complex(N, workloads.SEEDS["n14"])
    got = gpu_decompose(G, dtype, "xordiag")
    idx = workloads.sample_indices(N, workloads.SEEDS["n14_idx"])
    assert_close(got[idx.astype(np.int64)], oracle.decompose_at(ref_for(G, dtype), idx), G, dtype)


def test_n13_sampled_and_integer_exact():
    N = 13
    G = workloads.gaussian_complex(N, 1300)
    got = gpu_decompose(G, torch.complex128, "xordiag")
    idx = workloads.sample_indices(N, 1301, k=1024)
    assert_close(got[idx.astype(np.int64)], oracle.decompose_at(G, idx), G, torch.complex128)
    Gi = workloads.integer_complex(N, 1302)
    got = gpu_decompose(Gi, torch.complex128, "xordiag")
    np.testing.assert_array_equal(got[idx.astype(np.int64)], oracle.decompose_at(Gi, idx))


def test_n14_compose_reconstructs_sampled_entries():
    N = 14
    G = workloads.gaussian_complex(N, 1400)
    Gd = dev(G)
    back = host(pg.compose(pg.decompose(Gd)))
    rows = np.random.default_rng(1).integers(0, 1 << N, 4096)
    cols = np.random.default_rng(2).integers(0, 1 << N, 4096)
    assert np.max(np.abs(back[rows, cols] - G[rows, cols])) <= 4e-12 * maxabs(G)
    assert np.max(np.abs(back - G)) <= 4e-12 * maxabs(G)


def test_n15_kronecker_factorises():
    """G = A (x) B with A on the top 7 qubits: c[nA 4^8 + nB] = a[nA] b[nB] (any size)."""
    A = workloads.gaussian_complex(7, 1500)
    B = workloads.gaussian_complex(8, 1501)
    G = np.kron(A, B).astype(np.complex64)
    got = gpu_decompose(G, torch.complex64, "xordiag")
    del G
    a = oracle.decompose_full(A.astype(np.complex64).astype(np.complex128))
    rng = np.random.default_rng(1502)
    nA = rng.integers(0, 4 ** 7, 2048)
    nB = rng.integers(0, 4 ** 8, 2048)
    b = oracle.decompose_at(B.astype(np.complex64).astype(np.complex128), nB)
    want = a[nA] * b
    # the complex64 product A (x) B is rounded once; compare against the rounded input's terms
    err = np.max(np.abs(got[nA * 4 ** 8 + nB] - want))
    assert err <= 2e-6 * np.max(np.abs(A)) * np.max(np.abs(B))


# ------------------------------------------------------------- launch-shape variants --
@pytest.mark.parametrize("N", [6, 8, 11, 12, 13, 14])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_variants_agree_with_oracle(N, dtype):
    """Both XOR-diagonal launch shapes match the oracle; complex128 results are bit-identical
    across shapes (the transform is exact integer arithmetic)."""
    G = workloads.gaussian_complex(N, 900 + N)
    Gd = dev(G.astype(NP[dtype]))
    idx = workloads.sample_indices(N, 901, k=512)
    want = oracle.decompose_at(ref_for(G, dtype), idx)
    results = {}
    try:
        for v in ("unit8192", "unit4096", "unit4096x8", "unit8192x8"):
            ok = (v.startswith("unit8192") and 7 <= N <= 15) or (v.startswith("unit4096") and 6 <= N <= 14)
            if not ok:
                continue
            pg.set_variant(N, dtype, "decompose", v)
            pg.set_variant(N, dtype, "compose", v)
            c = pg.decompose(Gd, method="xordiag")
            results[v] = host(c)
            assert_close(results[v][idx.astype(np.int64)], want, G, dtype)
            back = host(pg.compose(c))
            assert np.max(np.abs(back - G.astype(NP[dtype]))) <= 4 * TOL[dtype] * maxabs(G)
    finally:
        pg.set_variant(N, dtype, "decompose", "default")
        pg.set_variant(N, dtype, "compose", "default")
    if dtype == torch.complex128 and len(results) > 1:
        first = next(iter(results.values()))
        for r in results.values():
            np.testing.assert_array_equal(r, first)


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_host_stream_pipeline_matches_per_matrix(dtype):
    """pauli_decompose_host_stream over 5 host matrices (two device buffer pairs, library
    streams): each output equals the single-matrix decomposition of its input, bit for bit."""
    N = 9
    mats = [workloads.gaussian_complex(N, 880 + k).astype(NP[dtype]) for k in range(5)]
    hosts = [torch.from_numpy(G).reshape(-1).pin_memory() for G in mats]
    outs = [torch.empty(4 ** N, dtype=dtype).pin_memory() for _ in mats]
    G_devs = [torch.empty(4 ** N, dtype=dtype, device="cuda") for _ in range(2)]
    out_devs = [torch.empty(4 ** N, dtype=dtype, device="cuda") for _ in range(2)]
    hosts_2d = [h.view(1 << N, 1 << N) for h in hosts]
    pg.pauli_decompose_host_stream(hosts_2d, outs, G_devs, out_devs)
    torch.cuda.synchronize()
    for G, o in zip(mats, outs):
        np.testing.assert_array_equal(o.numpy(), host(pg.decompose(dev(G))))


@pytest.mark.parametrize("N", [5, 8, 12, 13])
def test_transpose_flips_sign_of_odd_y_strings(N):
    """c_n(G^T) = (-1)^(number of Y factors) c_n(G): G^T has the same XOR-diagonals, each
    reversed by r -> r ^ x, which multiplies the transform by (-1)^popc(x & z). The fixed-point
    transform is exact, so the single-pass kernels agree bit for bit; the plain FP64 sum (N = 5)
    adds the same terms in another order, and the tiled kernel (N = 13) re-scales per tile, whose
    contents differ between G and G^T, so these agree to rounding."""
    G = workloads.gaussian_complex(N, 870 + N)
    a = host(pg.decompose(dev(G)))
    b = host(pg.decompose(dev(np.ascontiguousarray(G.T))))
    k = oracle.y_count(np.arange(4 ** N), N)
    want = np.where(k % 2 == 1, -1.0, 1.0) * a
    if 6 <= N <= 11:
        np.testing.assert_array_equal(b, want)
    else:  # N = 12, 13: the two-stage kernel is the default there
        assert np.max(np.abs(b - want)) <= 2 * TOL[torch.complex128] * maxabs(G)
