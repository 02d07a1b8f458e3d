"""GPU: pauli_decompose_batch_static, the batched decomposition that allocates nothing.

Callers that cannot allocate device memory -- a fixed memory budget, or an allocator that
must not be re-entered at that point -- use this entry point instead of a plan. It keeps its
work counter and matrix table in a fixed array in the library's device memory. These tests
call it through the C ABI twice in a row with different batches (the second call must not
see the first call's state) and compare every output with the existing entry points -- the
plan (same per-item arithmetic, bit for bit) and one launch per matrix (within the usual
tolerance, since small matrices there use the plain FP64 sum) -- and a seeded sample of each
matrix's coefficients with the CPU oracle. A captured call must replay its own batch: the
table travels as a kernel parameter, so a later direct call with another batch does not
change what the graph decomposes.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}
NP = {torch.complex128: np.complex128, torch.complex64: np.complex64}
CODE = {torch.complex128: 1, torch.complex64: 0}


def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def _static_enqueue(Gd, outs, Ns, dtype):
    lib = _lib.load()
    gp, k1 = _ptrs(Gd)
    op, k2 = _ptrs(outs)
    narr = (ctypes.c_int * len(Ns))(*[int(n) for n in Ns])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.pauli_decompose_batch_static(gp, narr, len(Ns), CODE[dtype], op, stream)
    assert st == 0, lib.pauli_last_error()


def _static_call(Gd, outs, Ns, dtype):
    _static_enqueue(Gd, outs, Ns, dtype)
    torch.cuda.synchronize()


def _check_oracle(mats, outs, dtype, seed):
    """A seeded sample of every matrix's coefficients against the CPU oracle (all of them for N <= 4)."""
    for b, (G, o) in enumerate(zip(mats, outs)):
        N = G.shape[0].bit_length() - 1
        idx = (np.arange(4 ** N, dtype=np.uint64) if N <= 4
               else workloads.sample_indices(N, seed * 7919 + b, k=48))
        ref = oracle.decompose_at(G, idx)
        got = o.cpu().numpy()[idx.astype(np.int64)]
        err = np.max(np.abs(got - ref))
        assert err <= TOL[dtype] * np.max(np.abs(G)), (b, N, err)


def _batch(seed, n, dtype):
    rng = np.random.default_rng(seed)
    Ns = rng.integers(1, 11, size=n)
    mats = [workloads.gaussian_complex(int(N), seed * 1000 + i).astype(NP[dtype]) for i, N in enumerate(Ns)]
    return Ns, mats


@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_static_batch_matches_existing_entry_points_twice(dtype):
    for seed, n in ((11, 37), (12, 64)):  # two calls in a row, different batches
        Ns, mats = _batch(seed, n, dtype)
        Gd = [torch.from_numpy(G).cuda() for G in mats]
        outs = [torch.full((4 ** int(N),), float("nan"), dtype=dtype, device="cuda") for N in Ns]
        _static_call(Gd, outs, Ns, dtype)
        # the same CTA shape as the static batch (512 threads), so that complex64 results,
        # whose rounding follows the order of the butterfly phases, match bit for bit
        plan = pg.PauliPlan([int(N) for N in Ns], dtype=dtype, threads_per_block=512)
        pouts = [torch.empty_like(o) for o in outs]
        plan.bind(Gd, pouts)
        plan.execute()
        assert plan.status() == 0
        sep = pg.decompose_list(Gd)
        torch.cuda.synchronize()
        for G, o, p, q in zip(mats, outs, pouts, sep):
            assert torch.equal(o, p)
            err = torch.max(torch.abs(o - q)).item()
            assert err <= TOL[dtype] * np.max(np.abs(G))
        _check_oracle(mats, outs, dtype, seed)


def test_static_batch_graph_replays_its_own_batch():
    """Capture one call, make a direct call with another batch, then replay: each output set must
    hold its own batch's coefficients (oracle sample), because the table is a kernel parameter."""
    dtype = torch.complex128
    NsA, matsA = _batch(21, 29, dtype)
    NsB, matsB = _batch(22, 41, dtype)
    GA = [torch.from_numpy(G).cuda() for G in matsA]
    GB = [torch.from_numpy(G).cuda() for G in matsB]
    outA = [torch.full((4 ** int(N),), float("nan"), dtype=dtype, device="cuda") for N in NsA]
    outB = [torch.full((4 ** int(N),), float("nan"), dtype=dtype, device="cuda") for N in NsB]
    _static_call(GB, outB, NsB, dtype)  # the first call on the device: before any capture
    for o in outB:
        o.fill_(float("nan"))
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        _static_enqueue(GA, outA, NsA, dtype)
    assert all(torch.isnan(o).all().item() for o in outA)  # capture enqueues nothing
    _static_call(GB, outB, NsB, dtype)  # a direct call with another table after the capture
    graph.replay()
    torch.cuda.synchronize()
    _check_oracle(matsA, outA, dtype, 21)
    _check_oracle(matsB, outB, dtype, 22)
    graph.replay()  # a second replay after nothing else: same result, bit for bit
    again = [o.clone() for o in outA]
    for o in outA:
        o.fill_(float("nan"))
    graph.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, o) for a, o in zip(again, outA))


def test_static_batch_rejects_oversized_batch():
    lib = _lib.load()
    n = 1025
    narr = (ctypes.c_int * n)(*([3] * n))
    null = (ctypes.c_void_p * n)()
    pp = ctypes.cast(null, ctypes.POINTER(ctypes.c_void_p))
    assert lib.pauli_decompose_batch_static(pp, narr, n, 1, pp, None) == 1  # PAULI_ERR_ARG, nothing launched
    assert b"1024" in lib.pauli_last_error()
