"""GPU: the project's autotuner end to end -- it times the launch-shape variants on the device,
writes a cache, the cache is applied through pauli_set_variant, the library reports the chosen
shapes, and decompositions under the tuned shapes still match the CPU oracle (complex128 results
are bit-identical across shapes: every shape runs the same exact integer transform)."""
import json

import numpy as np
import pytest
import torch

import oracle
import paper_2401_16378_gb300 as pg
from paper_2401_16378_gb300 import _lib, autotune, workloads

pytestmark = pytest.mark.gpu

OPS = ("decompose", "decompose_batched")


def test_tuner_times_variants_writes_and_applies_cache(tmp_path):
    lib = _lib.load()
    Ns = (8, 9)
    before = {(N, op): pg.get_variant(N, torch.complex128, op) for N in Ns for op in OPS}
    # the reference result of each N under the built-in shape
    mats = {N: workloads.gaussian_complex(N, 4400 + N) for N in Ns}
    ref = {N: pg.decompose(torch.from_numpy(G).cuda(), method="xordiag") for N, G in mats.items()}
    torch.cuda.synchronize()
    try:
        res = autotune.tune_variants(Ns=Ns, dtypes=("c128",), ops=OPS, reps=2)
        assert set(res) == {f"{N}/c128/{op}" for N in Ns for op in OPS}
        for key, rec in res.items():
            assert rec["best"] in (1, 2, 3, 4)  # the single-pass shapes exist for N = 8, 9
            assert len(rec["ms"]) >= 3 and all(v > 0 for v in rec["ms"].values())
            assert rec["ms"][str(rec["best"])] == min(rec["ms"].values())
        plan = autotune.tune_plan([3, 5, 8, 9, 9], dtypes=("c128",), reps=2)
        assert plan["c128"]["best_threads"] in (256, 512)
        path = tmp_path / "cache.json"
        path.write_text(json.dumps({"gpu": torch.cuda.get_device_name(0), "variants": res, "plan": plan}))
        # the tuner leaves the built-in shapes in place; applying the cache sets its choices
        for N in Ns:
            for op in OPS:
                assert lib.pauli_set_variant(N, _lib.PAULI_C128, autotune._OPS[op], 0) == 0
        assert autotune.apply_cached(str(path)) == len(res)
        for N in Ns:
            for op in OPS:
                assert pg.get_variant(N, torch.complex128, op) == res[f"{N}/c128/{op}"]["best"]
        for N, G in mats.items():
            Gd = torch.from_numpy(G).cuda()
            got = pg.decompose(Gd, method="xordiag")
            batch = pg.decompose(torch.stack([Gd, Gd]), method="xordiag")
            torch.cuda.synchronize()
            assert torch.equal(got, ref[N])
            assert torch.equal(batch[0], ref[N]) and torch.equal(batch[1], ref[N])
            idx = workloads.sample_indices(N, 4500 + N, k=256)
            err = np.max(np.abs(got.cpu().numpy()[idx.astype(np.int64)] - oracle.decompose_at(G, idx)))
            assert err <= 1e-12 * np.max(np.abs(G))
    finally:
        for (N, op), v in before.items():
            lib.pauli_set_variant(N, _lib.PAULI_C128, autotune._OPS[op], v)
