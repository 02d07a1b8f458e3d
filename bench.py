"""Benchmark of the dense Pauli decomposition on GB300 (one JSON line on rank 0).

Step: one decomposition of the N=14 workload -- a 16384 x 16384 complex128 matrix with
i.i.d. complex normal entries (seed 14) -- into all 4^14 Pauli coefficients by the
XOR-diagonal + Walsh-Hadamard kernel. Inputs (4 GiB) exceed the 129 MB L2, so no flush is
needed between steps. value = coefficients per second over the whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--n 14]

Under torchrun each rank decomposes its own copy of the workload (replicas: the path has
no exchange step); the time is the maximum over ranks.
`--impl reference` times the CPU oracle on the host cores on a bounded sample of the same
workload's coefficients (the tier's reference arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES = {"c128": 16, "c64": 8}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", "--qubits", dest="n", type=int, default=14, help="qubits of the timed workload")
    p.add_argument("--quick", action="store_true", help="skip the secondary forms")
    p.add_argument("--variant", default="default", choices=["default", "unit8192", "unit4096", "unit4096x8", "unit8192x8", "tiled8", "tiled16",
                            "twostage"],
                   help="XOR-diagonal launch shape of the timed step")
    p.add_argument("--profile", action="store_true",
                   help="only warm-up + timed kernel launches (for ncu); prints the step time")
    p.add_argument("--dtype", default="c128", choices=["c128", "c64"],
                   help="element type of the --profile launches (the timed step is complex128)")
    p.add_argument("--profile-batch", type=int, default=0,
                   help="with --profile: launch the batched plan over the first B matrices of the "
                        "uneven-N batch instead of the N-qubit decomposition")
    p.add_argument("--hermitian", action="store_true",
                   help="with --profile: the Hermitian form read from the upper triangle (real "
                        "output); with --profile-batch: the Hermitian plan")
    p.add_argument("--forms-only", default="",
                   help="comma list of secondary forms (n6, n12, c64, batched, adjoint, xhi, h14) to run alone, "
                        "without the timed step; prints their JSON")
    return p.parse_args()


# ------------------------------------------------------------------------------ helpers --
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash():
    h = hashlib.sha256()
    # the device code of the timed kernel (the two-stage twostage_kernel at N 12..14) and what it includes
    for name in ("twostage_impl.cuh", "ptx.cuh", "c64x.cuh", "twostage_c128.cu", "twostage_c64.cu", "tiled.h",
                 "xordiag_impl.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2401_16378_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(key):
    """DRAM bytes per launch from the committed ncu summary, if taken on the current source."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(key)
    except Exception:
        return None
    if not rec or rec.get("source_sha") != source_hash():
        return None
    return rec.get("bytes_per_launch")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        return time.time()

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        sm, mx, reasons = [], [], set()
        for ts, line in self.lines:
            if not (t0 <= ts <= t1):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_rate(G, N, seconds_target, seed=4242, impl=None):
    """Coefficients per second of a CPU implementation (default: the oracle) on a bounded random
    sample of the workload."""
    import oracle
    from paper_2401_16378_gb300 import workloads

    impl = impl or oracle
    threads = impl.default_threads()
    probe = workloads.sample_indices(N, seed, k=max(16, threads), with_special=False)
    t0 = time.perf_counter()
    impl.decompose_at(G, probe)
    dt = time.perf_counter() - t0
    k = len(probe)
    for attempt in range(3):  # the probe underestimates the rate (thread start-up): rescale once more
        k = int(max(len(probe), min(1 << 22, k * seconds_target / max(dt, 1e-6))))
        idx = workloads.sample_indices(N, seed + 1 + attempt, k=k, with_special=False)
        t0 = time.perf_counter()
        impl.decompose_at(G, idx)
        dt = time.perf_counter() - t0
        if dt >= 0.5 * seconds_target or k == 1 << 22:
            break
    return k / dt, k, dt, threads


def metric_name(N):
    return f"Pauli coefficients per second, N={N} complex128"


def workload_config(N, world):
    """The `config` object of both arms' JSON lines."""
    D = 1 << N
    return {"workload": f"N={N}: {D}x{D} complex128 dense matrix, i.i.d. complex normal entries "
                        f"(seed {14 if N == 14 else N}), all 4^{N} coefficients", "N": N,
            "matrix_bytes": 16 * 4 ** N, "l2": "inputs larger than L2 (no flush needed)", "io_dtype": "complex128",
            "parallelism": f"replicas x{world}"}


# --------------------------------------------------------------------------- reference arm --
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2401_16378_gb300 import workloads

    N = args.n
    G = workloads.gaussian_complex(N, workloads.SEEDS["n14"] if N == 14 else N)
    threads = oracle.default_threads()
    # one step = a bounded sample of the workload's coefficients (~1 s of host work)
    probe = workloads.sample_indices(N, 1, k=threads, with_special=False)
    t0 = time.perf_counter()
    oracle.decompose_at(G, probe)
    per = (time.perf_counter() - t0) / len(probe)
    k = max(threads, int(1.0 / max(per, 1e-9)))
    for w in range(args.warmup):
        oracle.decompose_at(G, workloads.sample_indices(N, 100 + w, k=threads, with_special=False))
    total_k, total_t = 0, 0.0
    for s in range(args.steps):
        idx = workloads.sample_indices(N, 1000 + s, k=k, with_special=False)
        t0 = time.perf_counter()
        oracle.decompose_at(G, idx)
        total_t += time.perf_counter() - t0
        total_k += k
    value = total_k / total_t
    sample = f"{k} seeded random coefficients of the N={N} matrix per step (O(2^N) each, Eq. (13))"
    line = {"impl": "reference", "metric": metric_name(N), "value": value,
            "unit": "coeffs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(N, world),
            "cpu_baseline": {"value": value, "unit": "coeffs/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "coeffs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------- multi-rank --
def max_over_ranks(ms: float, world: int, device) -> float:
    """The slowest rank's time (every rank gets it); the identity with one rank."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time.
    Ranks are replicas (each decomposes its own copy of the workload), so the units add up."""
    return world * units_per_rank / (ms * 1e-3)


# ------------------------------------------------------------------------------- our arm --
def event_time(fn, steps, stream):
    import torch

    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / steps  # ms


def run_ours(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    from paper_2401_16378_gb300 import _build

    _build.build()
    import paper_2401_16378_gb300 as pg
    from paper_2401_16378_gb300 import workloads

    if args.forms_only:
        only = set(args.forms_only.split(","))
        G14 = workloads.gaussian_complex(14, workloads.SEEDS["n14"]) if only & {"c64", "xhi"} else None
        forms = secondary_forms(pg, workloads, dev, torch.cuda.current_stream(dev), G14, only=only)
        print(json.dumps({"forms": forms}), flush=True)
        return

    N = args.n
    D = 1 << N
    ncoef = 4 ** N
    es = BYTES["c128"]
    G_h = workloads.gaussian_complex(N, workloads.SEEDS["n14"] if N == 14 else N)
    G = torch.from_numpy(G_h).to(dev)
    out = torch.empty(ncoef, dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream(dev)

    if args.variant != "default":
        pg.set_variant(N, torch.complex128, "decompose", args.variant)

    def step():
        pg.decompose(G, out=out, method="xordiag")

    if args.profile and args.profile_batch > 0:
        profile_plan(pg, workloads, dev, stream, args)
        return
    if args.profile:
        if args.dtype == "c64":
            G, out = G.to(torch.complex64), torch.empty(ncoef, dtype=torch.complex64, device=dev)
            if args.variant != "default":
                pg.set_variant(N, torch.complex64, "decompose", args.variant)
        if args.hermitian:
            out = torch.empty(ncoef, dtype=torch.float32 if args.dtype == "c64" else torch.float64, device=dev)

            def step():
                pg.decompose_hermitian(G, out=out, upper=True)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        ms = event_time(step, args.steps, stream)
        print(json.dumps({"profile": True, "N": N, "dtype": args.dtype, "hermitian_upper": args.hermitian,
                          "ms_per_step": ms}), flush=True)
        return

    def barrier():
        if world > 1:
            dist.barrier()

    sampler = ClockSampler(local if world > 1 else int(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0] or 0))
    with sampler:
        # warm-up inside the clock window: at least W steps and at least ~1 s of the same work,
        # so that the clock record spans many samples even when the timed region is short
        t_warm = time.time()
        n_warm = 0
        while n_warm < max(3, args.warmup) or time.time() - t_warm < 1.0:
            step()
            n_warm += 1
            if n_warm % 8 == 0:
                torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        t_start = time.time()
        ms = event_time(step, args.steps, stream)
        torch.cuda.synchronize(dev)
        t_end = time.time()
        barrier()
    clocks = sampler.summary(t_warm, t_end)
    clocks["window"] = f"{n_warm} warm-up steps and the {args.steps} timed steps"
    clocks["timed_region_samples"] = sampler.summary(t_start, t_end)["samples"]
    ms = max_over_ranks(ms, world, dev)
    value = aggregate_rate(ncoef, world, ms)

    # accuracy on sampled coefficients (oracle) -- rank 0
    res = {}
    if rank == 0:
        import oracle

        idx = workloads.sample_indices(N, workloads.SEEDS["n14_idx"] if N == 14 else 7, k=4096)
        got = out.cpu().numpy()[idx.astype(np.int64)]
        want = oracle.decompose_at(G_h, idx)
        res["max_err_over_max_abs_G"] = float(np.max(np.abs(got - want)) / np.max(np.abs(G_h)))
        res["sample"] = f"{idx.size} coefficients: 4096 seeded random indices and the special indices"
        res["tolerance_rel"] = 1e-12

    # end to end through the streaming host-buffer C ABI call: each step copies its matrix in
    # from pinned host memory, decomposes it and copies the coefficients back out; the library
    # pipelines consecutive steps over two device buffer sets (copy-in of step k + 1, compute of
    # step k and copy-out of step k - 1 at once).
    G_pin = torch.from_numpy(G_h).pin_memory()
    out_pins = [torch.empty(ncoef, dtype=torch.complex128).pin_memory() for _ in range(2)]
    G_devs, out_devs = [G.view(-1), torch.empty_like(G).view(-1)], [out, torch.empty_like(out)]
    e2e_steps = max(4, min(args.steps, 32))  # enough steps to amortise the pipeline fill and drain

    def e2e_run(k):
        pg.pauli_decompose_host_stream([G_pin] * k, [out_pins[i % 2] for i in range(k)], G_devs, out_devs,
                                       method="xordiag", stream=stream)

    e2e_run(2)  # the first call allocates the library streams and their scratch
    torch.cuda.synchronize(dev)
    barrier()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    e2e_run(e2e_steps)
    eb.record(stream)
    eb.synchronize()
    e2e_ms = ea.elapsed_time(eb) / e2e_steps
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    del G_pin, out_pins, G_devs, out_devs

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peak_hbm()
    alg_bytes = 2 * ncoef * es
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": recorded_traffic(f"xordiag N={N} c128"), "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes}

    rate, k, dt, cores = oracle_rate(G_h, N, seconds_target=12.0)
    cpu = {"value": rate, "unit": "coeffs/s", "cores": cores, "kind": "oracle",
           "sample": f"{k} seeded random coefficients of the N={N} workload in {dt:.1f} s (Eq. (13), O(2^N) each)"}
    from oracle import gray

    grate, gk, gdt, gcores = oracle_rate(G_h, N, seconds_target=8.0, impl=gray)
    cpu_gray = {"value": grate, "unit": "coeffs/s", "cores": gcores, "kind": "gray_code",
                "sample": f"{gk} seeded random coefficients of the N={N} workload in {gdt:.1f} s",
                "what": "the paper's CPU algorithm (Sec. 3): Eq. (13) in Gray-code order with the lambda recurrence "
                        "of Eq. (14), plain FP64 sums, C + OpenMP; a second, faster CPU baseline (not the checker)"}

    line = {"metric": metric_name(N), "value": value,
            "unit": "coeffs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": workload_config(N, world),
            "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_gray_code": cpu_gray,
            "e2e": {"value": aggregate_rate(ncoef, world, e2e_ms), "unit": "coeffs/s",
                    "h2d_bytes_per_step": ncoef * es, "d2h_bytes_per_step": ncoef * es, "ms_per_step": e2e_ms,
                    "steps": e2e_steps,
                    "mode": ("pauli_decompose_host_stream over the steps from pinned buffers: copy-in, decomposition "
                             "and copy-out of consecutive steps pipelined over two device buffer sets")},
            "gpu_launches": args.steps, "clocks": clocks, "accuracy": res}
    if not args.quick:
        line["forms"] = secondary_forms(pg, workloads, dev, stream, G_h if N == 14 else None)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def profile_plan(pg, workloads, dev, stream, args):
    """Warm-up + timed graph launches of the batched plan over the first B matrices of the
    512-matrix uneven-N batch (for ncu on a reduced batch); prints the launch time."""
    import torch

    tdt = torch.complex128 if args.dtype == "c128" else torch.complex64
    mats, Ns = workloads.batched_hermitian(workloads.SEEDS["batched"], batch=512)
    mats, Ns = mats[:args.profile_batch], [int(n) for n in Ns[:args.profile_batch]]
    rdt = torch.float64 if tdt == torch.complex128 else torch.float32
    Gd = [torch.from_numpy(G).to(dev).to(tdt) for G in mats]
    outs = [torch.empty(4 ** n, dtype=rdt if args.hermitian else tdt, device=dev) for n in Ns]
    plan = pg.PauliPlan(Ns, dtype=tdt, hermitian=args.hermitian)
    plan.bind(Gd, outs)
    for _ in range(args.warmup):
        plan.graph_launch()
    torch.cuda.synchronize(dev)
    ms = event_time(plan.graph_launch, args.steps, stream)
    st = plan.status()
    plan.close()
    ncoef = sum(4 ** n for n in Ns)
    print(json.dumps({"profile": True, "batch": len(Ns), "dtype": args.dtype, "hermitian": args.hermitian,
                      "coefficients": ncoef, "ms_per_launch": ms, "status": st}), flush=True)


def secondary_forms(pg, workloads, dev, stream, G14=None, only=None):
    """Plain, complex64, batched and adjoint forms on the same GPU, with their errors."""
    import torch

    import oracle

    forms = {}
    reps = 5

    def want(name):
        return only is None or name in only

    def timed(fn, n=reps):
        fn()
        torch.cuda.synchronize(dev)
        return event_time(fn, n, stream)

    if want("n6"):
        n6_form(pg, workloads, dev, oracle, timed, forms)
    if want("n12"):
        n12_forms(pg, workloads, dev, oracle, timed, forms)
    if want("c64") and G14 is not None:
        c64_form(pg, workloads, dev, oracle, timed, forms, G14)
    if want("batched"):
        batched_forms(pg, workloads, dev, oracle, timed, forms)
    if want("adjoint"):
        adjoint_form(pg, workloads, dev, oracle, timed, forms)
    if want("xhi") and G14 is not None:
        xhi_form(pg, workloads, dev, oracle, timed, forms, G14)
    if want("h14"):
        h14_form(pg, workloads, dev, oracle, timed, forms)
    return forms


def h14_form(pg, workloads, dev, oracle, timed, forms):
    """N=14 Hermitian complex128 matrix: real parts from the full matrix (24 B per coefficient)
    and from its upper triangle only (two-stage upper-triangle mode, 16 B per coefficient)."""
    import torch

    N = 14
    H = workloads.hermitian_complex(N, workloads.SEEDS["n12_herm"] + 2)
    h = torch.from_numpy(H).to(dev)
    r_full = torch.empty(4 ** N, dtype=torch.float64, device=dev)
    r_up = torch.empty_like(r_full)
    ms_full = timed(lambda: pg.decompose_hermitian(h, out=r_full), 10)
    ms_up = timed(lambda: pg.decompose_hermitian(h, out=r_up, upper=True), 10)
    same = bool(torch.equal(r_full, r_up))
    idx = workloads.sample_indices(N, 1414, k=512)
    err = float(np.max(np.abs(r_up.cpu().numpy()[idx.astype(np.int64)] - oracle.decompose_at(H, idx).real))
                / np.max(np.abs(H)))
    forms["n14_hermitian_real_c128"] = {"ms": ms_full, "coeffs_per_s": 4 ** N / (ms_full * 1e-3),
                                        "hbm_gbs_algorithmic": 4 ** N * 24 / (ms_full * 1e-3) / 1e9}
    forms["n14_hermitian_upper_c128"] = {"ms": ms_up, "coeffs_per_s": 4 ** N / (ms_up * 1e-3),
                                         "hbm_gbs_algorithmic": 4 ** N * 16 / (ms_up * 1e-3) / 1e9,
                                         "bit_identical_to_full_read": same, "max_err_rel": err,
                                         "sample": "512 seeded coefficients vs the oracle",
                                         "reads": "diagonal and upper triangle of G only"}
    del h, r_full, r_up


def xhi_form(pg, workloads, dev, oracle, timed, forms, G14):
    """x-class shards of the N=14 complex128 matrix on this one GPU: the block-XOR copy and the
    shard decomposition (2^k blocks of N - k qubits + the in-place k-bit combine) for shard 1."""
    import torch

    from paper_2401_16378_gb300 import shard

    N = 14
    g = torch.from_numpy(G14).to(dev)
    for k in (1, 3):
        L = torch.empty((1 << N, 1 << (N - k)), dtype=torch.complex128, device=dev)
        o = torch.empty(L.numel(), dtype=torch.complex128, device=dev)
        ms_layout = timed(lambda: pg.xhi_layout(g, k, 1, out=L), 10)
        ms = timed(lambda: pg.decompose_xhi(L, N, k, 1, out=o), 10)
        j = np.random.default_rng(1400 + k).integers(0, o.numel(), 1024)
        want = oracle.decompose_at(G14, shard.shard_indices(N, k, 1)[j])
        err = float(np.max(np.abs(o.cpu().numpy()[j] - want)) / np.max(np.abs(G14)))
        forms[f"n14_xhi_k{k}_c128"] = {
            "shards": 1 << k, "shard_ms": ms, "layout_copy_ms": ms_layout,
            "shard_coeffs_per_s": o.numel() / (ms * 1e-3),
            "hbm_gbs_algorithmic": 2 * o.numel() * 16 / (ms * 1e-3) / 1e9,
            "max_err_rel": err, "sample": "1024 seeded entries of shard 1 vs the oracle",
            "note": "one shard on one GPU; 2^k such shards make the N=14 decomposition"}
        del L, o
    del g


def n6_form(pg, workloads, dev, oracle, timed, forms):
    """N=6 config: plain kernel, latency."""
    import torch

    G6 = workloads.gaussian_complex(6, workloads.SEEDS["n6"])
    g6 = torch.from_numpy(G6).to(dev)
    o6 = torch.empty(4 ** 6, dtype=torch.complex128, device=dev)
    ms6 = timed(lambda: pg.decompose(g6, out=o6, method="plain"), 50)
    err6 = float(np.max(np.abs(o6.cpu().numpy() - oracle.decompose_full(G6))) / np.max(np.abs(G6)))
    # the same 50 calls captured in one CUDA graph: the kernel's own latency, without the
    # Python-side cost of each call
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        pg.decompose(g6, out=o6, method="plain")
    torch.cuda.current_stream(dev).wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for _ in range(50):
            pg.decompose(g6, out=o6, method="plain")
    ms6g = timed(graph.replay, 5) / 50
    forms["n6_plain_c128"] = {"us_per_call": ms6 * 1e3, "coeffs_per_s": 4 ** 6 / (ms6 * 1e-3), "max_err_rel": err6,
                              "graph_us_per_call": ms6g * 1e3,
                              "graph_coeffs_per_s": 4 ** 6 / (ms6g * 1e-3),
                              "note": "us_per_call: separate calls from Python; graph_: 50 calls in one CUDA graph"}
    del graph
    # the complex64 path on the same input (TwoSum-compensated FP32), error against the FP64 oracle
    # of the exactly upcast input
    G6s = G6.astype(np.complex64)
    g6s = torch.from_numpy(G6s).to(dev)
    o6s = torch.empty(4 ** 6, dtype=torch.complex64, device=dev)
    ms6s = timed(lambda: pg.decompose(g6s, out=o6s, method="plain"), 50)
    want6s = oracle.decompose_full(G6s.astype(np.complex128))
    forms["n6_plain_c64"] = {"us_per_call": ms6s * 1e3, "coeffs_per_s": 4 ** 6 / (ms6s * 1e-3),
                             "max_err_rel": float(np.max(np.abs(o6s.cpu().numpy() - want6s)) / np.max(np.abs(G6s))),
                             "tolerance_rel": 2e-6}


def n12_forms(pg, workloads, dev, oracle, timed, forms):
    """N=12 config: plain vs XOR-diagonal, general and Hermitian."""
    import torch

    N = 12
    for name, G in (("general", workloads.gaussian_complex(N, workloads.SEEDS["n12"])),
                    ("hermitian", workloads.hermitian_complex(N, workloads.SEEDS["n12_herm"]))):
        g = torch.from_numpy(G).to(dev)
        o = torch.empty(4 ** N, dtype=torch.complex128, device=dev)
        idx = workloads.sample_indices(N, workloads.SEEDS["n12_idx"])
        want = oracle.decompose_at(G, idx)
        for method, n in (("xordiag", 20), ("plain", 2)):
            ms = timed(lambda: pg.decompose(g, out=o, method=method), n)
            err = float(np.max(np.abs(o.cpu().numpy()[idx.astype(np.int64)] - want)) / np.max(np.abs(G)))
            entry = {"ms": ms, "coeffs_per_s": 4 ** N / (ms * 1e-3), "max_err_rel": err}
            if method == "plain":
                entry["fp64_adds_per_s"] = 2 * 8 ** N / (ms * 1e-3)
            else:
                entry["hbm_gbs_algorithmic"] = 2 * 4 ** N * 16 / (ms * 1e-3) / 1e9
            forms[f"n12_{name}_{method}_c128"] = entry
        if name == "hermitian":
            # real parts only (pauli_decompose_hermitian): 16 B read + 8 B written per coefficient
            r = torch.empty(4 ** N, dtype=torch.float64, device=dev)
            ms = timed(lambda: pg.decompose_hermitian(g, out=r), 20)
            err = float(np.max(np.abs(r.cpu().numpy()[idx.astype(np.int64)] - want.real)) / np.max(np.abs(G)))
            forms["n12_hermitian_xordiag_real_c128"] = {
                "ms": ms, "coeffs_per_s": 4 ** N / (ms * 1e-3), "max_err_rel": err,
                "hbm_gbs_algorithmic": 4 ** N * (16 + 8) / (ms * 1e-3) / 1e9,
                "max_abs_imag_dropped_rel": float(np.max(np.abs(want.imag)) / np.max(np.abs(G)))}
            # upper triangle only (pauli_decompose_hermitian_upper): 8 B read + 8 B written
            ms = timed(lambda: pg.decompose_hermitian(g, out=r, upper=True), 20)
            err = float(np.max(np.abs(r.cpu().numpy()[idx.astype(np.int64)] - want.real)) / np.max(np.abs(G)))
            forms["n12_hermitian_xordiag_upper_c128"] = {
                "ms": ms, "coeffs_per_s": 4 ** N / (ms * 1e-3), "max_err_rel": err,
                "hbm_gbs_algorithmic": 4 ** N * (8 + 8) / (ms * 1e-3) / 1e9,
                "reads": "diagonal and upper triangle of G only"}
            del r
        # the complex64 path on the same input, error against the FP64 oracle of the upcast input
        Gs = G.astype(np.complex64)
        gs = torch.from_numpy(Gs).to(dev)
        os_ = torch.empty(4 ** N, dtype=torch.complex64, device=dev)
        ms = timed(lambda: pg.decompose(gs, out=os_, method="xordiag"), 20)
        want_s = oracle.decompose_at(Gs.astype(np.complex128), idx)
        err = float(np.max(np.abs(os_.cpu().numpy()[idx.astype(np.int64)].astype(np.complex128) - want_s))
                    / np.max(np.abs(Gs)))
        forms[f"n12_{name}_xordiag_c64"] = {"ms": ms, "coeffs_per_s": 4 ** N / (ms * 1e-3), "max_err_rel": err,
                                            "hbm_gbs_algorithmic": 2 * 4 ** N * 8 / (ms * 1e-3) / 1e9,
                                            "tolerance_rel": 2e-6}
        del g, o, gs, os_
    # a real matrix (the general input's real part): 8 B read + 8 B written per coefficient
    Gr = np.ascontiguousarray(workloads.gaussian_complex(N, workloads.SEEDS["n12"]).real)
    gr = torch.from_numpy(Gr).to(dev)
    r = torch.empty(4 ** N, dtype=torch.float64, device=dev)
    ms = timed(lambda: pg.decompose_real(gr, out=r), 20)
    idx = workloads.sample_indices(N, workloads.SEEDS["n12_idx"])
    want = oracle.real_coefficients_at(Gr, idx)
    forms["n12_real_xordiag_c128"] = {
        "ms": ms, "coeffs_per_s": 4 ** N / (ms * 1e-3),
        "max_err_rel": float(np.max(np.abs(r.cpu().numpy()[idx.astype(np.int64)] - want)) / np.max(np.abs(Gr))),
        "hbm_gbs_algorithmic": 4 ** N * (8 + 8) / (ms * 1e-3) / 1e9,
        "input": "real part of the N=12 general matrix (float64)"}
    del gr, r


def c64_form(pg, workloads, dev, oracle, timed, forms, G14):
    """N=14 complex64 (TwoSum-compensated FP32): time and error against the FP64 oracle."""
    import torch

    N = 14
    G64 = G14.astype(np.complex64)
    g = torch.from_numpy(G64).to(dev)
    o = torch.empty(4 ** N, dtype=torch.complex64, device=dev)
    ms = timed(lambda: pg.decompose(g, out=o, method="xordiag"), 10)
    idx = workloads.sample_indices(N, workloads.SEEDS["n14_idx"])
    want = oracle.decompose_at(G64.astype(np.complex128), idx)
    got = o.cpu().numpy()[idx.astype(np.int64)].astype(np.complex128)
    forms["n14_xordiag_c64"] = {"ms": ms, "coeffs_per_s": 4 ** N / (ms * 1e-3),
                                "hbm_gbs_algorithmic": 2 * 4 ** N * 8 / (ms * 1e-3) / 1e9,
                                "max_err_rel": float(np.max(np.abs(got - want)) / np.max(np.abs(G64))),
                                "tolerance_rel": 2e-6}
    del g, o, G64
    # listed coefficients (pauli_coeffs_at, O(2^N) each, no scratch): the 4096 sampled indices
    # of the N=14 complex128 matrix
    g = torch.from_numpy(G14).to(dev)
    idx_d = torch.from_numpy(idx.astype(np.int64)).to(dev)
    oc = torch.empty(idx.size, dtype=torch.complex128, device=dev)
    ms = timed(lambda: pg.coeffs_at(g, idx_d, out=oc), 10)
    want = oracle.decompose_at(G14, idx)
    forms["n14_coeffs_at_c128"] = {
        "ms": ms, "coeffs": int(idx.size), "coeffs_per_s": idx.size / (ms * 1e-3),
        "gbs_read": idx.size * (1 << N) * 16 / (ms * 1e-3) / 1e9,
        "max_err_rel": float(np.max(np.abs(oc.cpu().numpy() - want)) / np.max(np.abs(G14))),
        "note": "each coefficient reads one XOR-diagonal of G (2^N elements, 16 B each) in the paper's per-coefficient form"}
    del g, idx_d, oc


def batched_forms(pg, workloads, dev, oracle, timed, forms):
    """512 Hermitian matrices, N uniform in 3..10, one persistent graph-captured launch against
    512 separate plain launches."""
    import torch

    mats, Ns = workloads.batched_hermitian(workloads.SEEDS["batched"], batch=512)
    Ns = [int(n) for n in Ns]
    ncoef = sum(4 ** n for n in Ns)
    rng = np.random.default_rng(5120)
    sel = [rng.integers(0, 4 ** n, 8) for n in Ns]
    for dname, tdt, npdt in (("c128", torch.complex128, np.complex128), ("c64", torch.complex64, np.complex64)):
        Gd = [torch.from_numpy(G.astype(npdt)).to(dev) for G in mats]
        outs = [torch.empty(4 ** n, dtype=tdt, device=dev) for n in Ns]
        plan = pg.PauliPlan(Ns, dtype=tdt)
        plan.bind(Gd, outs)
        ms_plan = timed(plan.graph_launch, 20)
        status = plan.status()
        errs = []
        for G, o, sl in zip(mats, outs, sel):
            Gr = G.astype(npdt).astype(np.complex128)
            got = o.cpu().numpy()[sl].astype(np.complex128)
            errs.append(np.max(np.abs(got - oracle.decompose_at(Gr, sl.astype(np.uint64)))) / np.max(np.abs(Gr)))
        plan.close()

        def separate():
            for g, o in zip(Gd, outs):
                pg.decompose(g, out=o, method="plain")

        ms_sep = timed(separate, 1)
        # the same batch as Hermitian matrices: upper triangles in, real coefficients out
        rdt = torch.float64 if tdt == torch.complex128 else torch.float32
        routs = [torch.empty(4 ** n, dtype=rdt, device=dev) for n in Ns]
        hplan = pg.PauliPlan(Ns, dtype=tdt, hermitian=True)
        hplan.bind(Gd, routs)
        ms_herm = timed(hplan.graph_launch, 20)
        herm_status = hplan.status()
        herm_err = 0.0
        for G, o, sl in zip(mats, routs, sel):
            Gr = G.astype(npdt).astype(np.complex128)
            got = o.cpu().numpy()[sl].astype(np.float64)
            herm_err = max(herm_err, float(np.max(np.abs(got - oracle.decompose_at(Gr, sl.astype(np.uint64)).real))
                                           / np.max(np.abs(Gr))))
        hplan.close()
        del routs
        forms[f"batched512_hermitian_{dname}"] = {
            "plan_graph_ms": ms_plan, "plan_coeffs_per_s": ncoef / (ms_plan * 1e-3), "plan_status": status,
            "hermitian_plan_graph_ms": ms_herm, "hermitian_plan_coeffs_per_s": ncoef / (ms_herm * 1e-3),
            "hermitian_plan_status": herm_status, "hermitian_plan_max_err_rel": herm_err,
            "hermitian_plan_speedup_vs_plain": ms_sep / ms_herm,
            "separate_plain_ms": ms_sep, "separate_plain_coeffs_per_s": ncoef / (ms_sep * 1e-3),
            "speedup_vs_plain": ms_sep / ms_plan, "max_err_rel": float(max(errs)),
            "sample": "8 seeded coefficients per matrix vs the oracle"}
        del Gd, outs


def adjoint_form(pg, workloads, dev, oracle, timed, forms):
    """64 matrices at N=10, loss = sum_n w_n |c_n|^2, forward + backward."""
    import torch

    N, B = 10, 64
    A = workloads.adjoint_inputs(workloads.SEEDS["adjoint"], batch=B, N=N)
    w_np = workloads.adjoint_weights(workloads.SEEDS["adjoint_w"], N)
    w = torch.from_numpy(w_np).to(dev)
    Gt = torch.from_numpy(A).to(dev).requires_grad_(True)

    def step_fused(method="xordiag"):
        # one fused kernel forward (decomposition + norm), one backward (weighted composition)
        Gt.grad = None
        loss, c = pg.decompose_weighted_norm_autograd(Gt, w, method=method)
        loss.backward()
        return c, loss

    def step_separate(torch_loss=False):
        Gt.grad = None
        c = pg.decompose_autograd(Gt, method="xordiag")
        loss = (w * c.abs() ** 2).sum() if torch_loss else pg.weighted_norm_autograd(c, w)
        loss.backward()
        return c, loss

    ms_x = timed(step_fused, 10)
    ms_s = timed(step_separate, 10)
    ms_t = timed(lambda: step_separate(torch_loss=True), 3)
    c, loss = step_fused()
    torch.cuda.synchronize(dev)
    ch = c.detach().cpu().numpy()
    want_loss = sum(oracle.weighted_norm(ch[k], w_np) for k in range(B))
    D = 1 << N
    rows = np.arange(0, D, 7)
    cols = (rows * 5 + 3) % D
    want = oracle.compose_at(oracle.weighted_norm_grad(ch[0], w_np), rows, cols) * 2.0 ** -N
    got = Gt.grad[0].cpu().numpy()[rows, cols]
    ms_p = timed(lambda: step_fused("plain"), 1)
    # the kernels of each step, each timed alone on the same buffers
    Gd = Gt.detach()
    cb = torch.empty_like(c)
    lb = torch.empty((), dtype=torch.float64, device=dev)
    gb = torch.empty_like(c)
    Ob = torch.empty_like(Gd)
    one = torch.ones(1, dtype=torch.float64, device=dev)
    parts = {"fused_decompose_norm_ms": timed(lambda: pg.decompose_weighted_norm(Gd, w, out=cb, loss=lb), 10),
             "fused_compose_weighted_ms": timed(lambda: pg.compose_weighted(cb, w, one, out=Ob, scale_exp=1 - N), 10),
             "decompose_ms": timed(lambda: pg.decompose(Gd, out=cb), 10),
             "weighted_norm_ms": timed(lambda: pg.weighted_norm(cb, w, out=lb), 10),
             "weighted_norm_grad_ms": timed(lambda: pg.weighted_norm_grad(cb, w, out=gb), 10),
             "compose_ms": timed(lambda: pg.compose(gb, out=Ob, scale_exp=-N), 10)}
    del cb, gb, Ob
    forms["adjoint64_n10_c128"] = {
        "fwd_bwd_ms": ms_x, "matrices_per_s": B / (ms_x * 1e-3), "coeffs_per_s": B * 4 ** N / (ms_x * 1e-3),
        "calls": "decompose_weighted_norm_autograd: fused decomposition + norm forward, weighted composition backward",
        "separate_kernels_fwd_bwd_ms": ms_s, "torch_elementwise_loss_fwd_bwd_ms": ms_t, "kernels_alone": parts,
        "plain_forward_fwd_bwd_ms": ms_p, "speedup_vs_plain": ms_p / ms_x,
        "hbm_gbs_algorithmic": 4 * B * 4 ** N * 16 / (ms_x * 1e-3) / 1e9,
        "loss_err_rel": abs(float(loss.detach().cpu()) - want_loss) / want_loss,
        "grad_max_err_rel": float(np.max(np.abs(got - want)) / np.max(np.abs(want))),
        "sample": "loss vs the oracle's norm of the 64 coefficient vectors; gradient of matrix 0 at 147 "
                  "entries vs the oracle's 2^-N compose of 2 w c"}
    del Gt
    # the same step in complex64 (TwoSum-compensated FP32), errors against the FP64 oracle
    A32 = A.astype(np.complex64)
    w32_np = w_np.astype(np.float32)
    w32 = torch.from_numpy(w32_np).to(dev)
    Gs = torch.from_numpy(A32).to(dev).requires_grad_(True)

    def step32():
        Gs.grad = None
        loss, c = pg.decompose_weighted_norm_autograd(Gs, w32)
        loss.backward()
        return c, loss

    ms32 = timed(step32, 10)
    c32, loss32 = step32()
    torch.cuda.synchronize(dev)
    c_ref = oracle.decompose_at(A32[0].astype(np.complex128), np.arange(4 ** N, dtype=np.uint64))
    c_err = float(np.max(np.abs(c32[0].detach().cpu().numpy().astype(np.complex128) - c_ref)) / np.max(np.abs(A32[0])))
    ch32 = c32.detach().cpu().numpy().astype(np.complex128)
    want_loss32 = sum(oracle.weighted_norm(ch32[k], w32_np.astype(np.float64)) for k in range(B))
    want32 = oracle.compose_at(oracle.weighted_norm_grad(ch32[0], w32_np.astype(np.float64)), rows, cols) * 2.0 ** -N
    got32 = Gs.grad[0].cpu().numpy()[rows, cols].astype(np.complex128)
    forms["adjoint64_n10_c64"] = {
        "fwd_bwd_ms": ms32, "matrices_per_s": B / (ms32 * 1e-3),
        "coeff_max_err_rel": c_err, "coeff_tolerance_rel": 2e-6,
        "loss_err_rel": abs(float(loss32.detach().cpu()) - want_loss32) / want_loss32,
        "grad_max_err_rel": float(np.max(np.abs(got32 - want32)) / np.max(np.abs(want32))),
        "sample": "coefficients of matrix 0 (all) vs the FP64 oracle of the upcast input; loss vs the oracle's "
                  "norm of the GPU coefficients; gradient of matrix 0 at 147 entries"}
    del Gs, A


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
