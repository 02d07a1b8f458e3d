"""GPU parity of the two-stage decompositions (PAULI_VARIANT_TILED8 / TILED16 / TWOSTAGE).

Stage 1 transforms 64 XY-masks x 64 rows per tile with a per-(class, tile) fixed-point
scale, stage 2 re-scales the tiles of each class to the class maximum and finishes the
transform. Checked against the oracle on sampled coefficients (random and special indices),
bit for bit on integer-valued inputs (every partial sum is exact on both sides, including
the re-scaling shift), on inputs whose tiles differ by many binades (the re-scaling path),
with all-zero tiles, with a non-finite entry, on a batch, and on repeated launches that reuse
the scratch ring. Tolerances as in test_gpu_parity: 1e-12 max|G| (complex128), 2e-6 max|G|
(complex64).
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
TILED = ("tiled8", "tiled16", "twostage")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def run_tiled(Gd, N, dtype, variant):
    pg.set_variant(N, dtype, "decompose", variant)
    try:
        c = pg.decompose(Gd, method="xordiag")
        pg.stream_status()
        return host(c)
    finally:
        pg.set_variant(N, dtype, "decompose", "default")


def assert_close(got, want, scale, dtype):
    err = np.max(np.abs(got.astype(np.complex128) - want))
    assert err <= TOL[dtype] * scale, f"err {err:.3e} > {TOL[dtype]:.0e} * {scale:.3e}"


@pytest.mark.parametrize("variant", TILED)
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
@pytest.mark.parametrize("N", [12, 13, 14])
def test_tiled_matches_oracle_and_single_pass(N, dtype, variant):
    G = workloads.gaussian_complex(N, 2000 + N)
    Gd = dev(G.astype(NP[dtype]))
    got = run_tiled(Gd, N, dtype, variant)
    idx = workloads.sample_indices(N, 2100 + N, k=1024)
    ref = G.astype(NP[dtype]).astype(np.complex128)
    assert_close(got[idx.astype(np.int64)], oracle.decompose_at(ref, idx), np.max(np.abs(G)), dtype)
    # every coefficient against the single-pass kernel (itself held to the oracle elsewhere)
    pg.set_variant(N, dtype, "decompose", "unit8192")
    try:
        single = host(pg.decompose(Gd, method="xordiag"))
    finally:
        pg.set_variant(N, dtype, "decompose", "default")
    assert_close(got, single.astype(np.complex128), 2 * np.max(np.abs(G)), dtype)


@pytest.mark.parametrize("variant", TILED)
@pytest.mark.parametrize("N", [12, 14])
def test_tiled_integer_input_bit_exact(N, variant):
    G = workloads.integer_complex(N, 2200 + N)
    got = run_tiled(dev(G), N, torch.complex128, variant)
    idx = workloads.sample_indices(N, 2300 + N, k=1024)
    np.testing.assert_array_equal(got[idx.astype(np.int64)], oracle.decompose_at(G, idx))


@pytest.mark.parametrize("variant", TILED)
def test_tiled_rescaling_across_binades_and_zero_tiles(variant):
    """Row blocks scaled by 2^e, e in [-60, 60], and some all-zero: each class's tiles sit at
    different fixed-point scales, and zero tiles carry exponent key 0."""
    N = 13
    G = workloads.gaussian_complex(N, 2400)
    rng = np.random.default_rng(2401)
    blocks = G.reshape(1 << (N - 6), 64, 1 << N)  # 64-row bands (tiles of both variants nest in them)
    e = rng.integers(-60, 61, size=blocks.shape[0])
    blocks *= (2.0 ** e)[:, None, None]
    blocks[rng.choice(blocks.shape[0], 9, replace=False)] = 0
    got = run_tiled(dev(G), N, torch.complex128, variant)
    idx = workloads.sample_indices(N, 2402, k=1024)
    assert_close(got[idx.astype(np.int64)], oracle.decompose_at(G, idx), np.max(np.abs(G)), torch.complex128)


@pytest.mark.parametrize("variant", ("tiled8", "twostage"))
def test_tiled_nonfinite_entry_gives_nan_for_its_mask_only(variant):
    N = 12
    G = workloads.gaussian_complex(N, 2500)
    G[700, 3001] = np.inf
    got = run_tiled(dev(G), N, torch.complex128, variant)
    n_all = np.arange(4 ** N, dtype=np.int64)
    even = np.zeros_like(n_all)
    odd = np.zeros_like(n_all)
    for t in range(N):
        even |= ((n_all >> (2 * t)) & 1) << t
        odd |= ((n_all >> (2 * t + 1)) & 1) << t
    mask = (even ^ odd) == (700 ^ 3001)
    assert np.all(np.isnan(got[mask]))
    assert not np.any(np.isnan(got[~mask]))


@pytest.mark.parametrize("variant", ("tiled8", "twostage"))
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_tiled_batch_and_repeated_launches(dtype, variant):
    """count = 3 matrices in one launch (blocks of later matrices reuse ring slots), then the
    same launch twice more: identical results every time."""
    N = 12
    Gs = np.stack([workloads.gaussian_complex(N, 2600 + b) for b in range(3)]).astype(NP[dtype])
    Gd = dev(Gs)
    pg.set_variant(N, dtype, "decompose_batched", variant)
    try:
        outs = [host(pg.decompose(Gd, method="xordiag")) for _ in range(3)]
        pg.stream_status()
    finally:
        pg.set_variant(N, dtype, "decompose_batched", "default")
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    idx = workloads.sample_indices(N, 2601, k=256)
    for b in range(3):
        ref = Gs[b].astype(np.complex128)
        assert_close(outs[0][b][idx.astype(np.int64)], oracle.decompose_at(ref, idx), np.max(np.abs(ref)), dtype)


def test_tiled_c64_unaligned_matrix_takes_single_pass_path():
    """A complex64 G that is 8- but not 16-byte aligned cannot feed the bulk copies; the call
    still succeeds (single-pass kernel) and matches the oracle."""
    N = 12
    G = workloads.gaussian_complex(N, 2700).astype(np.complex64)
    flat = torch.empty(4 ** N + 1, dtype=torch.complex64, device="cuda")
    flat[1:] = torch.from_numpy(G.ravel()).cuda()
    Gd = flat[1:].view(1 << N, 1 << N)
    assert Gd.data_ptr() % 16 == 8
    got = run_tiled(Gd, N, torch.complex64, "tiled8")
    idx = workloads.sample_indices(N, 2701, k=256)
    assert_close(got[idx.astype(np.int64)], oracle.decompose_at(G.astype(np.complex128), idx), np.max(np.abs(G)),
                 torch.complex64)


@pytest.mark.parametrize("variant", ("tiled16", "twostage"))
def test_tiled_bounded_wait_reports_timeout_and_recovers(variant):
    """The stall hook makes the producers of the next tiled launch wait on a count that nothing
    raises; the bounded wait gives up, the launch ends early, pauli_stream_status reports
    PAULI_ERR_TIMEOUT once, and the next launch on the same stream is correct again."""
    N = 12
    G = workloads.gaussian_complex(N, 2800)
    Gd = dev(G)
    pg.set_variant(N, torch.complex128, "decompose", variant)
    try:
        pg.debug_stall_next_tiled()
        pg.decompose(Gd, method="xordiag")
        with pytest.raises(pg.PauliError, match="TIMEOUT"):
            pg.stream_status()
        pg.stream_status()  # read once, then cleared
        got = host(pg.decompose(Gd, method="xordiag"))
        pg.stream_status()
    finally:
        pg.set_variant(N, torch.complex128, "decompose", "default")
    idx = workloads.sample_indices(N, 2801, k=256)
    assert_close(got[idx.astype(np.int64)], oracle.decompose_at(G, idx), np.max(np.abs(G)), torch.complex128)


def test_tiled_variant_is_decompose_only():
    with pytest.raises(pg.PauliError, match="UNSUPPORTED"):
        pg.set_variant(14, torch.complex128, "compose", "tiled8")
    with pytest.raises(pg.PauliError, match="UNSUPPORTED"):
        pg.set_variant(11, torch.complex128, "decompose", "tiled8")


def _workspace(N, dtype, count=1):
    nbytes = pg.decompose_workspace_size(N, count, dtype)
    assert nbytes > 0
    return torch.empty(nbytes, dtype=torch.uint8, device="cuda")


@pytest.mark.parametrize("variant", ("tiled16", "twostage"))
@pytest.mark.parametrize("N", [12, 13])
def test_decompose_ws_matches_library_workspace(N, variant):
    """Caller-provided scratch gives the same bits as the library's per-stream buffer."""
    dtype = torch.complex128
    G = workloads.gaussian_complex(N, 3100 + N)
    Gd = dev(G)
    pg.set_variant(N, dtype, "decompose", variant)
    try:
        ws = _workspace(N, dtype)
        a = pg.decompose_ws(Gd, ws, method="xordiag")
        pg.workspace_status(ws)
        b = pg.decompose(Gd, method="xordiag")
        pg.stream_status()
        torch.cuda.synchronize()
        assert torch.equal(a, b)
        with pytest.raises(pg.PauliError, match="ERR_ARG"):
            pg.decompose_ws(Gd, ws[: ws.numel() - 256], method="xordiag")  # too small: rejected, nothing runs
    finally:
        pg.set_variant(N, dtype, "decompose", "default")
    idx = workloads.sample_indices(N, 3200 + N, k=256)
    assert_close(host(a)[idx.astype(np.int64)], oracle.decompose_at(G, idx), np.max(np.abs(G)), dtype)


@pytest.mark.parametrize("variant", ("tiled16", "twostage"))
def test_decompose_ws_first_call_on_a_stream_under_graph_capture(variant):
    """With caller scratch nothing is allocated, so the first tiled call on a fresh stream can be
    captured; the graph replays it."""
    N, dtype = 12, torch.complex128
    G = workloads.gaussian_complex(N, 3300)
    Gd = dev(G)
    pg.set_variant(N, dtype, "decompose", variant)
    try:
        want = pg.decompose(Gd, method="xordiag")  # kernel set-up outside the capture
        pg.stream_status()
        ws = _workspace(N, dtype)
        out = torch.full_like(want, float("nan"))
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        with torch.cuda.graph(graph, stream=side):
            pg.decompose_ws(Gd, ws, out=out, method="xordiag")
        assert torch.isnan(out).all().item()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, want)
        pg.workspace_status(ws)
    finally:
        pg.set_variant(N, dtype, "decompose", "default")


def test_release_workspaces_then_decompose_again():
    N, dtype = 12, torch.complex128
    G = workloads.gaussian_complex(N, 3400)
    Gd = dev(G)
    s = torch.cuda.Stream()
    pg.set_variant(N, dtype, "decompose", "tiled16")
    try:
        with torch.cuda.stream(s):
            a = pg.decompose(Gd, method="xordiag")
            pg.release_workspaces()  # frees this stream's ring after synchronising it
            b = pg.decompose(Gd, method="xordiag")  # allocates afresh
            pg.stream_status()
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    finally:
        pg.set_variant(N, dtype, "decompose", "default")


@pytest.mark.parametrize("N", [13, 14])
def test_two_stage_variants_agree_bit_for_bit_in_complex128(N):
    """The three two-stage kernels run the same int64 transform with the same per-tile scales:
    identical complex128 coefficients."""
    G = workloads.gaussian_complex(N, 3500 + N)
    Gd = dev(G)
    outs = [run_tiled(Gd, N, torch.complex128, v) for v in TILED]
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


def _class_of_all(N):
    n_all = np.arange(4 ** N, dtype=np.int64)
    even = np.zeros_like(n_all)
    odd = np.zeros_like(n_all)
    for t in range(N):
        even |= ((n_all >> (2 * t)) & 1) << t
        odd |= ((n_all >> (2 * t + 1)) & 1) << t
    return even ^ odd


@pytest.mark.parametrize("N,variant", [(12, "twostage"), (10, None)])
@pytest.mark.parametrize("bad", [1e36, np.inf])
def test_complex64_out_of_range_entry_gives_nan_for_its_mask_only(N, variant, bad):
    """A complex64 value beyond the compensated grid's range (above about 2^(126 - N)) or a
    non-finite one makes every coefficient of its XY-mask NaN and leaves the others exact."""
    D = 1 << N
    G = workloads.gaussian_complex(N, 2600 + N).astype(np.complex64)
    r, q = 700 % D, 3001 % D
    G[r, q] = np.complex64(bad)
    Gd = dev(G)
    if variant:
        got = run_tiled(Gd, N, torch.complex64, variant)
    else:
        got = host(pg.decompose(Gd, method="xordiag"))
    mask = _class_of_all(N) == (r ^ q)
    assert np.all(np.isnan(got[mask]))
    assert not np.any(np.isnan(got[~mask]))
    idx = workloads.sample_indices(N, 2601, k=512)
    idx = idx[~mask[idx.astype(np.int64)]]
    Gc = G.astype(np.complex128)
    Gc[r, q] = 0  # the other masks never read the entry
    assert_close(got[idx.astype(np.int64)], oracle.decompose_at(Gc, idx), np.max(np.abs(Gc)), torch.complex64)
