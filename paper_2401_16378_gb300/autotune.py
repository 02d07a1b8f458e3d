"""Autotuner for libpauli's launch shapes.

The XOR-diagonal kernels come in several launch shapes (include/pauli.h, PAULI_VARIANT_*):
8192-element work units on 512-thread CTAs (one per SM) or 4096-element units on 256-thread
CTAs (two per SM), with 16 or 8 elements per thread, which differ in how the N butterfly
stages split between registers, shared memory and the CTA cluster; and, for decomposition
at N 12..14, the two-stage tiled kernel with either CTA size. The batched plan has the same two CTA shapes. Which is
faster depends on N, the dtype and the direction, so this module times each candidate on a
seeded synthetic input with CUDA events, keeps the fastest, applies it with
pauli_set_variant, and stores the choices in a JSON cache keyed by the GPU's name.

    python -m paper_2401_16378_gb300.autotune [--out PATH] [--n 6 7 ... 14]

When the library is first loaded the package applies the cache named by
$PAULI_AUTOTUNE_CACHE, else the file autotune_cache.json next to this module, when its GPU
name matches the current device ($PAULI_AUTOTUNE=0 turns this off).
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np
import torch

from . import _lib

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")
_DT = {"c128": torch.complex128, "c64": torch.complex64}
_DT_CODE = {"c128": _lib.PAULI_C128, "c64": _lib.PAULI_C64}
_OPS = {"decompose": 0, "compose": 1, "decompose_batched": 2, "compose_batched": 3}
BATCH_ELEMENTS = 1 << 26  # a tuning batch holds about this many elements (1 GiB of complex128)
VARIANT_RANGE = {1: (7, 15), 2: (6, 14), 3: (6, 14), 4: (7, 15), 5: (12, 14), 6: (12, 14),
                 7: (12, 14)}  # variant -> N range
DECOMPOSE_ONLY = {5, 6, 7}  # the two-stage variants


def _gpu_name() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _time(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def tune_variants(Ns=range(6, 15), dtypes=("c128", "c64"), ops=tuple(_OPS), reps=5, seed=777):
    """Time every variant for each (N, dtype, op); returns {"N/dtype/op": {"best": v, "ms": {...}}}.
    The "_batched" ops time a batch of max(2, BATCH_ELEMENTS / 4^N) matrices."""
    from . import api

    lib = _lib.load()
    out = {}
    for N in Ns:
        D = 1 << N
        rng = np.random.default_rng(seed + N)
        for dt in dtypes:
            tdt = _DT[dt]
            # one matrix; a batch repeats it (one buffer pair serves as matrix/coefficients)
            one = torch.from_numpy((rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))).astype(
                np.complex128)).to(tdt).cuda()
            for op in ops:
                count = max(2, BATCH_ELEMENTS >> (2 * N)) if op.endswith("_batched") else 1
                a = one.expand(count, D, D).contiguous()
                b = torch.empty_like(a)
                times = {}
                for v, (lo, hi) in VARIANT_RANGE.items():
                    if not lo <= N <= hi or (op.startswith("compose") and v in DECOMPOSE_ONLY):
                        continue
                    _lib.check(lib.pauli_set_variant(N, _DT_CODE[dt], _OPS[op], v))
                    if op.startswith("decompose"):
                        times[v] = _time(lambda: api.pauli_decompose(a, out=b.view(count, -1), method="xordiag"),
                                         reps)
                    else:
                        times[v] = _time(lambda: api.pauli_compose(a.view(count, -1), out=b), reps)
                _lib.check(lib.pauli_set_variant(N, _DT_CODE[dt], _OPS[op], 0))
                del a, b
                if times:
                    best = min(times, key=times.get)
                    out[f"{N}/{dt}/{op}"] = {"best": best, "count": count,
                                             "ms": {str(k): v for k, v in times.items()}}
            del one
            torch.cuda.empty_cache()
    return out


def tune_plan(Ns, dtypes=("c128", "c64"), reps=5, seed=778):
    """Time the batched plan with 512- and 256-thread CTAs for the list of N."""
    from . import api

    rng = np.random.default_rng(seed)
    res = {}
    for dt in dtypes:
        tdt = _DT[dt]
        mats = [torch.from_numpy((rng.standard_normal((1 << n, 1 << n)) + 1j * rng.standard_normal(
            (1 << n, 1 << n))).astype(np.complex128)).to(tdt).cuda() for n in Ns]
        outs = [torch.empty(4 ** n, dtype=tdt, device="cuda") for n in Ns]
        times = {}
        for threads in (512, 256):
            plan = api.PauliPlan(Ns, dtype=tdt, threads_per_block=threads)
            plan.bind(mats, outs)
            times[threads] = _time(plan.graph_launch, reps)
            plan.close()
        res[dt] = {"best_threads": min(times, key=times.get), "ms": {str(k): v for k, v in times.items()}}
    return res


def apply(cache: dict) -> int:
    """Apply cached variant choices to libpauli; returns how many were applied."""
    lib = _lib.load()
    n = 0
    for key, rec in cache.get("variants", {}).items():
        N, dt, op = key.split("/")
        if lib.pauli_set_variant(int(N), _DT_CODE[dt], _OPS[op], int(rec["best"])) == 0:
            n += 1
    return n


def load_cache(path: str | None = None) -> dict | None:
    path = path or os.environ.get("PAULI_AUTOTUNE_CACHE") or DEFAULT_CACHE
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def apply_cached(path: str | None = None) -> int:
    """Apply the cache if it was measured on a GPU of the current device's name."""
    cache = load_cache(path)
    if not cache or not torch.cuda.is_available() or cache.get("gpu") != _gpu_name():
        return 0
    return apply(cache)


def plan_threads(dtype: torch.dtype) -> int:
    """Tuned CTA size for batched plans (0 = library default)."""
    cache = load_cache()
    if not cache or not torch.cuda.is_available() or cache.get("gpu") != _gpu_name():
        return 0
    dt = "c64" if dtype == torch.complex64 else "c128"
    return int(cache.get("plan", {}).get(dt, {}).get("best_threads", 0))


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--out", default=DEFAULT_CACHE)
    p.add_argument("--n", type=int, nargs="*", default=list(range(6, 15)))
    p.add_argument("--reps", type=int, default=5)
    args = p.parse_args()
    data = {"gpu": _gpu_name(), "variants": tune_variants(args.n, reps=args.reps)}
    from . import workloads

    _, Ns = workloads.batched_hermitian(workloads.SEEDS["batched"], batch=512)
    data["plan"] = tune_plan([int(n) for n in Ns], reps=args.reps)
    with open(args.out, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    print(json.dumps(data))


if __name__ == "__main__":
    main()
