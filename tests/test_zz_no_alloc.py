"""GPU: pauli_decompose_batch_static, the batched decomposition that allocates nothing.

Callers that cannot allocate device memory -- a fixed memory budget, or an allocator that
must not be re-entered at that point -- use this entry point instead of a plan. It keeps its
work counter and matrix table in a fixed array in the library's device memory. This test
calls it through the C ABI twice in a row with different batches (the second call must not
see the first call's state) and compares every output with the existing entry points: the
plan (same per-item arithmetic, bit for bit) and one launch per matrix (within the usual
tolerance, since small matrices there use the plain FP64 sum).
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import _lib, workloads

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}
NP = {torch.complex128: np.complex128, torch.complex64: np.complex64}
CODE = {torch.complex128: 1, torch.complex64: 0}


def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)), arr


def _static_call(Gd, outs, Ns, dtype):
    lib = _lib.load()
    gp, k1 = _ptrs(Gd)
    op, k2 = _ptrs(outs)
    narr = (ctypes.c_int * len(Ns))(*[int(n) for n in Ns])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.pauli_decompose_batch_static(gp, narr, len(Ns), CODE[dtype], op, stream)
    assert st == 0, lib.pauli_last_error()
    torch.cuda.synchronize()


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


def test_static_batch_rejects_oversized_batch():
    lib = _lib.load()
    n = 1025
    narr = (ctypes.c_int * n)(*([3] * n))
    null = (ctypes.c_void_p * n)()
    pp = ctypes.cast(null, ctypes.POINTER(ctypes.c_void_p))
    assert lib.pauli_decompose_batch_static(pp, narr, n, 1, pp, None) == 1  # PAULI_ERR_ARG, nothing launched
    assert b"1024" in lib.pauli_last_error()
