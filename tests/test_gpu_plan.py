"""GPU: the persistent batched plan (uneven N, one launch, graph replay) against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = {torch.complex128: 1e-12, torch.complex64: 2e-6}
NP = {torch.complex128: np.complex128, torch.complex64: np.complex64}


def _check(mats, outs, dtype, rng, per=24):
    for G, o in zip(mats, outs):
        N = G.shape[0].bit_length() - 1
        got = o.cpu().numpy()
        Gr = G.astype(NP[dtype]).astype(np.complex128)
        if N <= 5:
            want, sel = oracle.decompose_full(Gr), np.arange(4 ** N)
        else:
            sel = rng.integers(0, 4 ** N, per)
            want = oracle.decompose_at(Gr, sel)
        err = np.max(np.abs(got[sel] - want))
        assert err <= TOL[dtype] * np.max(np.abs(G)), (N, err)


@pytest.mark.parametrize("threads", [512, 256])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_batched_config_graph_replay(threads, dtype):
    mats, Ns = workloads.batched_hermitian(workloads.SEEDS["batched"], batch=512)
    Gd = [torch.from_numpy(G.astype(NP[dtype])).cuda() for G in mats]
    outs = [torch.full((4 ** int(n),), float("nan"), dtype=dtype, device="cuda") for n in Ns]
    plan = pg.PauliPlan(Ns, dtype=dtype, threads_per_block=threads)
    plan.bind(Gd, outs)
    plan.graph_launch()
    assert plan.status() == 0
    _check(mats, outs, dtype, np.random.default_rng(5))
    first = [o.clone() for o in outs]
    for o in outs:
        o.fill_(float("nan"))
    plan.graph_launch()  # replay
    assert plan.status() == 0
    for a, b in zip(first, outs):
        assert torch.equal(a, b)
    # the same bits as one XOR-diagonal launch per matrix (both exact integer transforms;
    # below N=6 the single-matrix path is the plain FP64 sum, checked against the oracle above)
    if dtype == torch.complex128:
        for G, o, n in zip(Gd, outs, Ns):
            if n >= 6:
                assert torch.equal(pg.decompose(G, method="xordiag"), o)


def test_plan_small_only_and_execute():
    Ns = [1, 2, 3, 4, 5, 6]
    mats = [workloads.gaussian_complex(n, 50 + n) for n in Ns]
    Gd = [torch.from_numpy(G).cuda() for G in mats]
    outs = [torch.empty(4 ** n, dtype=torch.complex128, device="cuda") for n in Ns]
    plan = pg.PauliPlan(Ns)
    plan.bind(Gd, outs)
    plan.execute()
    assert plan.status() == 0
    _check(mats, outs, torch.complex128, np.random.default_rng(6))


def test_plan_bounded_wait_reports_timeout():
    """The stall hook makes block 0 wait on a flag nothing sets; the wait gives up after a
    bounded number of polls, the status word reads PAULI_ERR_TIMEOUT, and the results are
    still complete (the other blocks took the work)."""
    Ns = [8, 7, 6]
    mats = [workloads.gaussian_complex(n, 70 + n) for n in Ns]
    Gd = [torch.from_numpy(G).cuda() for G in mats]
    outs = [torch.empty(4 ** n, dtype=torch.complex128, device="cuda") for n in Ns]
    plan = pg.PauliPlan(Ns)
    plan.bind(Gd, outs)
    plan.set_stall(True)
    plan.execute()
    assert plan.status() == 8  # PAULI_ERR_TIMEOUT
    assert "bounded wait" in pg.last_error()
    _check(mats, outs, torch.complex128, np.random.default_rng(7))
    plan.set_stall(False)
    plan.execute()
    assert plan.status() == 0


# ---------------------------------------------------------------------- Hermitian plans --
@pytest.mark.parametrize("threads", [512, 256])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_hermitian_plan_batched_config(threads, dtype):
    """The batched config (512 Hermitian matrices, N 3..10) through a Hermitian plan: real
    coefficients from the upper triangles, against the oracle and, in complex128 bit for bit,
    against pauli_decompose_hermitian_upper of each matrix (both exact integer transforms of
    the same upper-triangle data; below N = 7 the single-matrix path is the plain FP64 sum)."""
    mats, Ns = workloads.batched_hermitian(workloads.SEEDS["batched"], batch=512)
    Gd = [torch.from_numpy(G.astype(NP[dtype])).cuda() for G in mats]
    rdt = torch.float64 if dtype == torch.complex128 else torch.float32
    outs = [torch.full((4 ** int(n),), float("nan"), dtype=rdt, device="cuda") for n in Ns]
    plan = pg.PauliPlan(Ns, dtype=dtype, threads_per_block=threads, hermitian=True)
    plan.bind(Gd, outs)
    plan.graph_launch()
    assert plan.status() == 0
    rng = np.random.default_rng(7)
    for G, o in zip(mats, outs):
        N = G.shape[0].bit_length() - 1
        Gr = G.astype(NP[dtype]).astype(np.complex128)
        sel = np.arange(4 ** N) if N <= 5 else rng.integers(0, 4 ** N, 24)
        want = oracle.decompose_at(Gr, sel.astype(np.uint64)).real
        err = np.max(np.abs(o.cpu().numpy()[sel].astype(np.float64) - want))
        assert err <= TOL[dtype] * np.max(np.abs(G)), (N, err)
    if dtype == torch.complex128:
        for G, o, n in zip(Gd, outs, Ns):
            if n >= 7:
                assert torch.equal(pg.decompose_hermitian(G, upper=True), o), n


def test_hermitian_plan_ignores_lower_triangle():
    Ns = [3, 6, 7, 9, 10, 5, 8]
    mats = [workloads.hermitian_complex(n, 60 + n) for n in Ns]
    bad = []
    for G in mats:
        B = G.copy()
        B[np.tril_indices(G.shape[0], -1)] = np.nan
        B.imag[np.diag_indices(G.shape[0])] = np.nan
        bad.append(B)
    res = []
    for src in (mats, bad):
        Gd = [torch.from_numpy(G).cuda() for G in src]
        outs = [torch.empty(4 ** n, dtype=torch.float64, device="cuda") for n in Ns]
        plan = pg.PauliPlan(Ns, dtype=torch.complex128, threads_per_block=256, hermitian=True)
        plan.bind(Gd, outs)
        plan.execute()
        assert plan.status() == 0
        res.append([o.cpu().numpy() for o in outs])
        plan.close()
    for a, b in zip(*res):
        np.testing.assert_array_equal(a, b)
        assert np.all(np.isfinite(b))
