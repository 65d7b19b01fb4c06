#!/usr/bin/env python
"""Benchmark of the filtered Paterson-Stockmeyer evaluator on one GB300.

Workload (default): Z = -0.5 * (5-point Dirichlet Laplacian on a 128 x 128
grid), n = 16384, nnz = 81408, ||Z||_1 = 4, FP64 CSR; one step evaluates
exp(Z) and cos(Z) with eps_tol = 1e-12 (Algorithm 2, filtered).  The metric
is evaluations per second (each step counts 2), with p50/p99 latency per
evaluation.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl psf|reference]

With --gpus N > 1 (launched by torchrun) each rank evaluates its own copy:
the evaluations are independent, so ranks are replicas with no collective
on the data path (weak scaling).  `--impl reference` times the CPU oracle
(the plain FP64 restatement of the paper's algorithm) on the host cores.
Prints one JSON line on rank 0.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "filtered-PS evals/s, HBM GB/s vs dense-PS on GB300 @relerr<=1e-12; p50/p99 ms"
WORKLOAD = "lap2d_128x128"
KINDS = ("exp", "cos")
TOL = 1e-12
# FP64 peak of the GB300 FP64 pipe: 152 SMs x 2 FMA/clk/SM x 2 flop x 2.07 GHz
FP64_UNITS = 152 * 2 * 2  # SMs x fma per clock per SM x flop per fma
FP64_PEAK_TFLOPS = FP64_UNITS * 2.07e9 / 1e12
PROFILE_JSON = os.path.join(ROOT, "profiles", "k_product_traffic.json")


def hbm_peak_gbs() -> float:
    """Measured HBM copy bandwidth (MEASURED_PEAKS.json, when present), else 6800 GB/s."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0
KERNEL_SOURCES = [os.path.join(ROOT, "paper_2208_05683_gb300", "csrc", f)
                  for f in ("psf_kernels.cu", "psf_device.cuh")]


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def job_rate(units_per_rank: float, local_ms: float, world: int, device=None):
    """Whole-job rate over replicas: the units all ranks processed divided by
    the slowest rank's time (max over ranks); returns (rate, max ms)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_ms = float(t.item())
    return world * units_per_rank / (local_ms / 1e3), local_ms


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []  # (host time of the sample, fields)
        self.proc = None
        self.thread = None
        self.window = None  # (t0, t1): the timed region

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.perf_counter(), parts))

    def mark(self, t0: float, t1: float):
        """The timed region, in time.perf_counter() seconds."""
        self.window = (t0, t1)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        rows = [r for t, r in self.rows]
        if self.window is not None:
            # samples taken while the timed region ran (a sample arrives up to
            # one period after it was taken)
            t0, t1 = self.window
            rows = [r for t, r in self.rows if t0 <= t <= t1 + 0.05]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        self_rows = rows

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[1]) for r in self_rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in self_rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self_rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self_rows)}


def config_dict(n: int, nnz: int, world: int) -> dict:
    """The workload's config, the same in both arms."""
    return {"workload": f"{WORKLOAD} exp+cos tol {TOL:g}", "n": n, "nnz": nnz, "evals_per_step": len(KINDS),
            "l2": "flushed before each step (256 MB write)", "parallelism": f"replicas x{world}"}


def fp64_probe(L, stream_ptr, gpu_index: int):
    """The library's FP64 rate probe (psf_fp64_peak: 8 independent fma chains
    per thread, 4 x 256 threads per SM), with the SM clock sampled while it
    runs: the probe draws the most power of anything here, and a clock held
    below its maximum by the power limit lowers its rate with it."""
    import ctypes
    cs = ClockSampler(gpu_index)
    cs.start()
    time.sleep(0.3)  # nvidia-smi's first sample
    t0 = time.perf_counter()
    v = ctypes.c_double()
    rc = L.psf_fp64_peak(stream_ptr, ctypes.byref(v))
    cs.mark(t0, time.perf_counter())
    cs.stop()
    clk = cs.summary()
    return {"tflops": v.value if rc == 0 else None, "sm_mhz": clk["sm_mhz"], "reasons": clk["reasons"],
            "nominal_at_probe_clock": (FP64_UNITS * clk["sm_mhz"] * 1e6 / 1e12) if clk["sm_mhz"] else None}


def fp64_peak(clock_mhz):
    """The FP64 pipe's rate at the SM clock of the timed region: 152 SMs x
    2 fma per clock x 2 flop (the unit count; the probe reaches 99.9 % of it
    at 2070 MHz)."""
    mhz = clock_mhz or 2070.0
    return FP64_UNITS * mhz * 1e6 / 1e12, f"FP64 pipe: 152 SMs x 2 fma/clk x 2 flop x {mhz:.0f} MHz (timed region)"


def _oracle_eval_worker(task):
    """One oracle evaluation in a worker process (the CPU baseline on all cores)."""
    import oracle
    import synthetic as syn
    rp, col, val, kind = task
    t0 = time.perf_counter()
    oracle.psscf(oracle.CSR(len(rp) - 1, rp, col, val), syn.coeffs(kind), TOL)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(rp, col, val):
    """The oracle as it stands on every host core: one evaluation per worker
    process (exp and cos alternating), evaluations being independent; the
    rate is evaluations over the wall time once the workers are up."""
    import concurrent.futures as cf
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=ctx) as ex:
        list(ex.map(_noop, range(cores)))  # workers started and imports done
        tasks = [(rp, col, val, KINDS[i % len(KINDS)]) for i in range(cores)]
        t0 = time.perf_counter()
        per = list(ex.map(_oracle_eval_worker, tasks))
        dt = time.perf_counter() - t0
    return {"value": cores / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} evaluations of the full {WORKLOAD} workload (exp and cos alternating), one per "
                      f"worker process, {dt:.1f} s wall; single evaluation median {statistics.median(per):.2f} s"}


def _noop(x):
    import oracle  # noqa: F401
    import synthetic  # noqa: F401
    return x


def make_inputs():
    import synthetic as syn
    rp, col, val = syn.workload(WORKLOAD)[0]
    return rp, col, val


def cpu_baseline(rp, col, val, evals_kinds=KINDS):
    """The oracle as it stands, one evaluation of each kind, single thread."""
    import oracle
    import synthetic as syn
    Z = oracle.CSR(len(rp) - 1, rp, col, val)
    t0 = time.perf_counter()
    for kind in evals_kinds:
        oracle.psscf(Z, syn.coeffs(kind), TOL)
    dt = time.perf_counter() - t0
    return {"value": len(evals_kinds) / dt, "unit": "evals/s", "cores": 1, "kind": "oracle",
            "sample": f"one exp and one cos evaluation of the full {WORKLOAD} workload ({dt:.1f} s)"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    rp, col, val = make_inputs()
    import oracle
    import synthetic as syn
    Z = oracle.CSR(len(rp) - 1, rp, col, val)
    coeffs = {k: syn.coeffs(k) for k in KINDS}
    for _ in range(args.warmup):
        for k in KINDS:
            oracle.psscf(Z, coeffs[k], TOL)
    lat = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for k in KINDS:
            t1 = time.perf_counter()
            oracle.psscf(Z, coeffs[k], TOL)
            lat.append((time.perf_counter() - t1) * 1e3)
    dt = time.perf_counter() - t0
    value = args.steps * len(KINDS) / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": config_dict(Z.n, Z.nnz, world),
        "p50_ms": statistics.median(lat), "p99_ms": sorted(lat)[min(len(lat) - 1, int(0.99 * len(lat)))],
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps of exp+cos on the full workload"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_psf(args):
    import ctypes
    import numpy as np
    import torch

    import paper_2208_05683_gb300 as psf
    import synthetic as syn
    from paper_2208_05683_gb300 import _abi

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    L = psf.lib()
    stream = torch.cuda.current_stream()

    rp, col, val = make_inputs()
    n = len(rp) - 1
    Z = psf.DeviceCSR.from_host(rp, col, val, device=dev)
    series = {k: psf.Series(syn.coeffs(k), TOL, kernel=args.kernel) for k in KINDS}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def one_step(lat=None, ser=series):
        out = []
        for k in KINDS:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = ser[k].eval_handle(Z, stream)
            e1.record(stream)
            out.append((h, e0, e1))
        for h, e0, e1 in out:
            e1.synchronize()
            if lat is not None:
                lat.append(e0.elapsed_time(e1))
            _abi.check(L.psf_result_destroy(h))

    # the product kernel's slot-map crossover, timed on this workload (outside
    # the timed region; results do not depend on it)
    tuned = None
    if not args.no_autotune:
        c, saved = psf.autotune(series[KINDS[0]], Z)
        tuned = {"table_crossover": c if c < 1e299 else "never", "saved_ms_per_eval": saved}

    # clocks sampled from before the warm-up (nvidia-smi takes a moment to
    # start); only the samples taken during the timed region are kept
    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(args.warmup):
        one_step()

    # ---- timed region: K steps, L2 flushed before each
    cnt0 = ctypes_i64(L.psf_launch_count)
    barrier()
    t_region = time.perf_counter()
    lat = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        one_step(lat)
    barrier()
    clocks.mark(t_region, time.perf_counter())
    clocks.stop()
    launches = ctypes_i64(L.psf_launch_count) - cnt0
    evals = args.steps * len(KINDS)
    value, total_ms = job_rate(evals, sum(lat), world, dev)

    # ---- roofline of the product kernel (event-timed launches, separate pass)
    _abi.check(L.psf_profile(1))
    for _ in range(2):
        flush.zero_()
        torch.cuda.synchronize()
        one_step()
    nl, ms, fma = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _abi.check(L.psf_profile_read(ctypes.byref(nl), ctypes.byref(ms), ctypes.byref(fma), 1))
    _abi.check(L.psf_profile(0))
    achieved = 2.0 * fma.value / (ms.value / 1e3) / 1e12
    clk = clocks.summary()
    peak, peak_source = fp64_peak(clk["sm_mhz"])
    probe = fp64_probe(L, ctypes.c_void_p(stream.cuda_stream), local) if rank == 0 else None
    traffic = None
    try:
        prof = json.load(open(PROFILE_JSON))
        if prof.get("kernel_hash") == kernel_hash() and prof.get("workload") == WORKLOAD:
            traffic = prof.get("dram_bytes_per_launch")
    except (OSError, ValueError):
        pass
    # DRAM rate of the product kernel: ncu bytes per launch x launches / event-timed duration
    dram_gbs = traffic * nl.value / (ms.value / 1e3) / 1e9 if traffic and ms.value > 0 else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": "k_product",
                "dram_gbs": dram_gbs, "dram_frac_of_hbm": dram_gbs / hbm_peak_gbs() if dram_gbs else None,
                "peak_source": peak_source, "fp64_probe": probe,
                "launches_timed": nl.value, "kernel_ms": ms.value, "algorithmic_fma": fma.value}

    # ---- end to end through the C ABI on host buffers: psf_eval_from_host
    # (pinned host Z copied in by the library) and psf_result_copy into
    # pinned host arrays, both evaluations, copies inside the timed region.
    # Each result is copied out on a second stream once its evaluation is
    # done, so the first result's copy runs while the second evaluation
    # computes; the step ends when both copies have landed.
    pin = [torch.as_tensor(x).pin_memory() for x in (np.asarray(rp, np.int32), np.asarray(col, np.int32),
                                                      np.asarray(val, np.float64))]
    zs_host = _abi.CSRStruct(n, int(len(col)), pin[0].data_ptr(), pin[1].data_ptr(), pin[2].data_ptr())
    h2d = sum(t.numel() * t.element_size() for t in pin)
    e2e_ms, d2h = [], 0
    # pinned host result arrays, allocated in the warm-up steps
    host_buf = {}

    def host_arrays(k, nnz):
        want = {"rowptr": (n + 1, torch.int32), "col": (max(nnz, 1), torch.int32), "val": (max(nnz, 1), torch.float64)}
        for name, (cnt, dt) in want.items():
            b = host_buf.get((k, name))
            if b is None or b.numel() < cnt:
                host_buf[(k, name)] = torch.empty(cnt, dtype=dt, pin_memory=True)
        return [host_buf[(k, name)] for name in ("rowptr", "col", "val")]

    st_ptr = ctypes.c_void_p(stream.cuda_stream)
    copy_stream = torch.cuda.Stream(device=dev)
    cp_ptr = ctypes.c_void_p(copy_stream.cuda_stream)
    for it in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        copy_stream.wait_event(e0)
        handles, copied = [], 0
        for k in KINDS:
            h = ctypes.c_void_p()
            _abi.check(L.psf_eval_from_host(series[k]._h, ctypes.byref(zs_host), st_ptr, ctypes.byref(h)))
            info = _abi.InfoStruct()
            _abi.check(L.psf_result_info(h, ctypes.byref(info)))
            hr, hc, hv = host_arrays(k, int(info.nnz))
            done = torch.cuda.Event()
            done.record(stream)
            copy_stream.wait_event(done)
            _abi.check(L.psf_result_copy(h, ctypes.c_void_p(hr.data_ptr()), ctypes.c_void_p(hc.data_ptr()),
                                         ctypes.c_void_p(hv.data_ptr()), cp_ptr))
            copied += (n + 1) * 4 + int(info.nnz) * 12
            handles.append(h)
        landed = torch.cuda.Event()
        landed.record(copy_stream)
        stream.wait_event(landed)
        e1.record(stream)
        e1.synchronize()
        for h in handles:
            _abi.check(L.psf_result_destroy(h))
        if it >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
            d2h = copied
    e2e_value, _ = job_rate(len(KINDS) * len(e2e_ms), sum(e2e_ms), world, dev)

    # ---- dense FP64 PS on the same GPU, run for real (same plan), with its
    # accuracy against the closed form beside the sparse result's
    dense = None
    if not args.no_dense and rank == 0:
        dense = measure_dense_ps(args, dev)

    # ---- the same workload with ||Z^2||..||Z^10|| estimated (PSF_Z_ESTIMATE)
    # instead of computed from the powers: an option's cost, not the headline
    est = None
    if rank == 0 and world == 1 and not args.no_estimate:
        est_series = {k: psf.Series(syn.coeffs(k), TOL, kernel=args.kernel, estimate=True) for k in KINDS}
        for _ in range(args.warmup):
            one_step(ser=est_series)
        elat = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            one_step(elat, ser=est_series)
        plans, ratios = {}, []
        for k in KINDS:
            ie, ix = est_series[k].eval(Z).info, series[k].eval(Z).info
            plans[k] = {key: [ie[key], ix[key]] for key in ("N", "q", "b", "products")}
            ratios += [ie["z"][i] / ix["z"][i] for i in range(2, 11) if ix["z"][i] > 0]
        est = {"evals_per_s": len(elat) / (sum(elat) / 1e3), "p50_ms": statistics.median(elat),
               "plans_equal": all(v[0] == v[1] for p in plans.values() for v in p.values()),
               "plans_estimate_vs_exact": plans, "z_estimate_over_exact_min": min(ratios) if ratios else None,
               "how": "same steps and timing as the headline, series created with estimate=True"}

    square = None
    if rank == 0 and world == 1 and not args.no_square:
        square = measure_square(args, Z, flush)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(rp, col, val)
        cpu["all_cores"] = cpu_baseline_all_cores(rp, col, val)
    batched = serving = sweep = None
    if rank == 0 and world == 1 and not args.no_sweep:
        sweep = measure_tol_sweep(args, dev)
    if rank == 0 and world == 1 and not args.no_batched:
        batched = measure_batched(args, dev, flush)
    if rank == 0 and world == 1 and not args.no_serving:
        serving = measure_serving(args, dev)

    if rank == 0:
        lat_sorted = sorted(lat)
        line = {
            "metric": METRIC, "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(n, int(len(col)), world),
            "kernel": args.kernel, "autotune": tuned,
            "p50_ms": statistics.median(lat_sorted),
            "p99_ms": lat_sorted[min(len(lat_sorted) - 1, int(0.99 * len(lat_sorted)))],
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clk,
            "dense_ps": dense,
            "batched": batched,
            "serving": serving,
            "tol_sweep": sweep,
            "z_estimate": est,
            "z_square": square,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def lap1d_closed_form(m: int, kind: str):
    """f(A) for A = -0.5 tridiag(-1, 2, -1) (m x m) through its sine eigenbasis:
    A = V diag(-(1 - cos(k pi / (m + 1)))) V with V the orthonormal DST-I
    matrix; kind exp, cos or sin."""
    import numpy as np
    k = np.arange(1, m + 1)
    V = np.sqrt(2.0 / (m + 1)) * np.sin(np.outer(k, k) * np.pi / (m + 1))
    lam = -(1.0 - np.cos(k * np.pi / (m + 1)))
    f = {"exp": np.exp, "cos": np.cos, "sin": np.sin}[kind](lam)
    return (V * f) @ V


def dense_ps(Zd, a, N: int, q: int, b: int):
    """Unfiltered Paterson-Stockmeyer (Eqs. 2-4) on dense FP64 matrices with
    torch.matmul: powers Z^2..Z^q, S_0 = B_{b-1}, S_i = B_{b-1-i} + Z^q S_{i-1},
    B_i = sum_j a_{iq+j} Z^j (a_k = 0 for k >= N)."""
    import torch
    n = Zd.shape[0]
    P = [torch.eye(n, dtype=torch.float64, device=Zd.device), Zd]
    for _ in range(2, q + 1):
        P.append(Zd @ P[-1])

    def block(i):
        B = torch.zeros_like(Zd)
        for j in range(q):
            if i * q + j < N and a[i * q + j] != 0.0:
                B.add_(P[j], alpha=a[i * q + j])
        return B

    S = block(b - 1)
    for i in range(1, b):
        S = block(b - 1 - i) + P[q] @ S
    return S


def measure_dense_ps(args, dev):
    """Dense FP64 PS (torch.matmul, cuBLAS) with the sparse scheme's own plan
    (N, q, b) on the 2D Laplacian: event-timed at 64 x 64 (n = 4096, the same
    plan as the 128 x 128 workload, ||Z||_1 = 4), with the 1-norm errors of the
    dense and of the filtered sparse result against the closed form
    exp/cos(A + B) of the Kronecker sum; the workload's n = 16384 projected by
    n^3 (or run with --dense-full); and the 1D Laplacian n = 256 the same way."""
    import numpy as np
    import torch
    import paper_2208_05683_gb300 as psf
    import synthetic as syn

    def dense_of(csr, n):
        rp, col, val = (torch.as_tensor(np.asarray(x)).to(dev) for x in csr)
        rows = torch.repeat_interleave(torch.arange(n, device=dev), (rp[1:] - rp[:-1]).long())
        X = torch.zeros(n, n, dtype=torch.float64, device=dev)
        X[rows, col.long()] = val.double()
        return X

    def rel1(X, F):
        return float(torch.linalg.matrix_norm(X - F, ord=1) / torch.linalg.matrix_norm(F, ord=1))

    def timed_dense(Zd, a, p, reps=2):
        dense_ps(Zd, a, p["N"], p["q"], p["b"])  # warm-up
        ms = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            D = dense_ps(Zd, a, p["N"], p["q"], p["b"])
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return D, min(ms)

    def case(host, n, exact, kind):
        a = syn.coeffs(kind)
        Z = psf.DeviceCSR.from_host(*host, device=dev)
        s = psf.Series(a, TOL)
        s.eval(Z)
        r = s.eval(Z)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(3):
            r = s.eval(Z)
        torch.cuda.synchronize()
        sparse_ms = (time.perf_counter() - t0) / 3 * 1e3
        p = r.info
        Zd = dense_of(host, n)
        D, dense_ms = timed_dense(Zd, a, p)
        F = exact.to(dev)
        out = {"n": n, "kind": kind, "N": p["N"], "q": p["q"], "b": p["b"], "dense_ms": dense_ms,
               "dense_evals_per_s": 1e3 / dense_ms, "sparse_ms": sparse_ms, "speedup_sparse": dense_ms / sparse_ms,
               "dense_err_1": rel1(D, F), "sparse_err_1": rel1(dense_of(r.csr.to_host(), n), F),
               "dense_density": float((D != 0).sum()) / n / n}
        del D, Zd, F
        torch.cuda.empty_cache()
        return out

    rows = []
    m = 64
    e1 = {k: torch.as_tensor(lap1d_closed_form(m, k)) for k in ("exp", "cos", "sin")}
    exact2d = {"exp": torch.kron(e1["exp"], e1["exp"]),
               "cos": torch.kron(e1["cos"], e1["cos"]) - torch.kron(e1["sin"], e1["sin"])}
    for kind in KINDS:
        rows.append(case(syn.laplacian_2d(m), m * m, exact2d[kind], kind))
    rows.append(case(syn.laplacian_1d(256), 256, torch.as_tensor(lap1d_closed_form(256, "exp")), "exp"))
    full = None
    if args.dense_full:
        M = 128
        E = torch.as_tensor(lap1d_closed_form(M, "exp"))
        full = case(syn.laplacian_2d(M), M * M, torch.kron(E, E), "exp")
    per_kind = [r for r in rows if r["n"] == m * m]
    proj_ms = sum(r["dense_ms"] for r in per_kind) / len(per_kind) * (128 * 128 / (m * m)) ** 3
    return {"rows": rows, "full_size": full, "evals_per_s": 1e3 / proj_ms if full is None else 1e3 / full["dense_ms"],
            "measured_at_full_size": full is not None,
            "projected_n16384_ms": proj_ms,
            "how": "dense PS run with torch.matmul float64 and the sparse plan's N, q, b; errors are relative "
                   "1-norm errors against the closed form of the 2D/1D Laplacian; n = 16384 projected from "
                   "n = 4096 by n^3 unless --dense-full"}


def measure_batched(args, dev, flush):
    """The batched workload: 512 instances (n log-uniform in [64, 4096], 1D/2D
    Laplacian or banded, ||Z||_1 in [1, 4], exp or cosh, tol 1e-12) in one
    psf_eval_batch call, against the same instances evaluated one by one."""
    import ctypes
    import torch
    import paper_2208_05683_gb300 as psf
    import synthetic as syn
    from paper_2208_05683_gb300 import _abi
    L = psf.lib()
    stream = torch.cuda.current_stream()
    inst = syn.batch_instances(512)
    series = [psf.Series(syn.coeffs(k), tol) for _, k, tol in inst]
    Zs = [psf.DeviceCSR.from_host(*Z, device=dev) for Z, _, _ in inst]
    count = len(Zs)
    sh = (ctypes.c_void_p * count)(*[x._h.value for x in series])
    zs = (_abi.CSRStruct * count)(*[z._struct() for z in Zs])
    sp = ctypes.c_void_p(stream.cuda_stream)

    def once():
        outs = (ctypes.c_void_p * count)()
        _abi.check(L.psf_eval_batch(sh, zs, count, sp, outs))
        for i in range(count):
            _abi.check(L.psf_result_destroy(ctypes.c_void_p(outs[i])))

    for _ in range(3):
        once()
    # the library's batch autotuner on these instances: slot-map crossover
    # per size class of work per row, row bitmaps, baby-step reuse
    tune = None
    if not args.no_autotune:
        bt = _abi.BatchTune()
        _abi.check(L.psf_autotune_batch(sh, zs, count, sp, ctypes.byref(bt)))
        tune = bt.as_dict()
        if tune["table_crossover"] >= 1e300:
            tune["table_crossover"] = "never"
    reps, ms = 5, []
    c0 = ctypes_i64(L.psf_launch_count)
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        once()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    launches = (ctypes_i64(L.psf_launch_count) - c0) / reps
    _abi.check(L.psf_profile(1))
    once()
    torch.cuda.synchronize()
    nl, pms, fma = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _abi.check(L.psf_profile_read(ctypes.byref(nl), ctypes.byref(pms), ctypes.byref(fma), 1))
    _abi.check(L.psf_profile(0))
    # the same instances one psf_eval at a time
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for x, z in zip(series, Zs):
        _abi.check(L.psf_result_destroy(x.eval_handle(z, stream)))
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    med = statistics.median(ms)
    return {"instances": count, "rows": int(sum(z.n for z in Zs)), "nnz": int(sum(z.nnz for z in Zs)),
            "inst_per_s": count / (med / 1e3), "ms_per_batch": med, "launches_per_batch": launches,
            "product_tflops": 2.0 * fma.value / (pms.value / 1e3) / 1e12 if pms.value > 0 else None,
            "algorithmic_fma": fma.value, "autotune": tune,
            "sequential_inst_per_s": count / t_seq, "speedup_vs_sequential": (count / (med / 1e3)) / (count / t_seq),
            "how": "median of 5 event-timed psf_eval_batch calls (L2 flushed before each), inputs resident"}


def measure_serving(args, dev):
    """Serving: a Poisson stream of requests (n log-uniform in [256, 65536],
    1D/2D Laplacian or banded, exp/cos/sinh, tol from {1e-8, 1e-10, 1e-12})
    through the library's server at 0.7x its measured saturated rate."""
    import numpy as np
    import torch
    import paper_2208_05683_gb300 as psf
    import synthetic as syn
    count = args.serving_requests
    reqs = syn.serving_requests(count, seed0=0)
    series = [psf.Series(syn.coeffs(k), tol) for _, k, tol in reqs]
    Zs = [psf.DeviceCSR.from_host(*Z, device=dev) for Z, _, _ in reqs]
    workers, max_batch = 4, 16
    srv = psf.Server(workers=workers, max_batch=max_batch)
    try:
        def drain(k):
            got = []
            while len(got) < k:
                got += srv.poll(256, 100, take=False)
            return got

        for i in range(min(24, count)):  # warm-up: pool sizes, kernels
            srv.submit(series[i], Zs[i], i)
        drain(min(24, count))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(count):
            srv.submit(series[i], Zs[i], i)
        drain(count)
        sat = count / (time.perf_counter() - t0)
        rate = 0.7 * sat
        rng = np.random.default_rng(1)
        gaps = rng.exponential(1.0 / rate, count)
        done = []
        t_start = time.perf_counter()
        t_next = t_start
        for i in range(count):
            t_next += gaps[i]
            while True:
                now = time.perf_counter()
                if now >= t_next:
                    break
                done += srv.poll(256, int(max(0.0, (t_next - now) * 1e3)), take=False)
            srv.submit(series[i], Zs[i], count + i)
        done += drain(count - len(done))
        t_end = time.perf_counter()
        stats = srv.stats()
    finally:
        srv.close()
    lat = sorted(c["latency_ms"] for c in done)
    return {"requests": count, "rate_per_s": rate, "evals_per_s": count / (t_end - t_start),
            "p50_ms": statistics.median(lat), "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "saturated_evals_per_s": sat, "mean_batch": float(np.mean([c["batch_size"] for c in done])),
            "max_concurrent": stats["max_concurrent"], "failed": stats["failed"], "workers": workers,
            "max_batch": max_batch,
            "sample": f"{count} requests (seeds 0..{count - 1}) of the serving mixture; Poisson arrivals at 0.7x "
                      "the saturated rate measured on the same requests",
            "latency": "host clock, submit to result available"}


def run_size_sweep(args):
    """The bench's 2D Laplacian on larger grids (exp, tol 1e-12): evaluation
    time (median of 5, event-timed, L2 flushed before each), and the product
    kernel's achieved FP64 rate over all its launches (library event timing),
    per grid size.  The per-row latency of the product kernel is amortised
    over more rows per warp as n grows."""
    import ctypes
    import torch
    import paper_2208_05683_gb300 as psf
    import synthetic as syn
    from paper_2208_05683_gb300 import _abi
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    L = psf.lib()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    rows = []
    for m in (128, 256, 384, 512, 768):
        Z = psf.DeviceCSR.from_host(*syn.laplacian_2d(m), device=dev)
        s = psf.Series(syn.coeffs("exp"), TOL)
        for _ in range(2):
            s.eval(Z)
        lat = []
        for it in range(5):
            flush.zero_()
            torch.cuda.synchronize()
            if it == 4:
                _abi.check(L.psf_profile(1))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h = s.eval_handle(Z, stream)
            e1.record(stream)
            e1.synchronize()
            _abi.check(L.psf_result_destroy(h))
            lat.append(e0.elapsed_time(e1))
        nl, ms, fma = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
        _abi.check(L.psf_profile_read(ctypes.byref(nl), ctypes.byref(ms), ctypes.byref(fma), 1))
        _abi.check(L.psf_profile(0))
        tf = 2.0 * fma.value / (ms.value / 1e3) / 1e12
        rows.append({"grid": m, "n": m * m, "ms": statistics.median(lat), "evals_per_s": 1e3 / statistics.median(lat),
                     "product_tflops": tf, "product_frac": tf / FP64_PEAK_TFLOPS, "product_ms": ms.value,
                     "fma": fma.value})
        print(f"{m}x{m}: {rows[-1]['ms']:.2f} ms, product kernel {tf:.3f} TFLOP/s "
              f"({100 * tf / FP64_PEAK_TFLOPS:.1f} %)", file=sys.stderr, flush=True)
    print(json.dumps({"experiment": "lap2d m x m, exp, tol 1e-12", "rows": rows}), flush=True)


def measure_tol_sweep(args, dev):
    """The banded workload (n = 65536, half-bandwidth 5, ||Z||_1 = 2, exp)
    over tolerances 1e-8..1e-14: time, result density and products per
    evaluation, against dense FP64 PS on the same GPU (products x one
    measured n x n float64 matmul, projected from n = 8192 by n^3 since
    three dense 65536^2 matrices would hold 100 GB)."""
    import torch
    import paper_2208_05683_gb300 as psf
    import synthetic as syn
    rp, col, val = syn.banded_random(65536, 5, 0, 2.0)
    n = len(rp) - 1
    Z = psf.DeviceCSR.from_host(rp, col, val, device=dev)
    m = 8192
    A = torch.randn(m, m, dtype=torch.float64, device=dev)
    torch.matmul(A, A)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    torch.matmul(A, A)
    e1.record()
    e1.synchronize()
    t_gemm = e0.elapsed_time(e1) / 1e3 * (n / m) ** 3
    del A
    torch.cuda.empty_cache()
    rows = []
    for tol in (1e-8, 1e-9, 1e-10, 1e-11, 1e-12, 1e-13, 1e-14):
        s = psf.Series(syn.coeffs("exp"), tol)
        for _ in range(2):
            s.eval(Z)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            r = s.eval(Z)
        torch.cuda.synchronize()
        t = (time.perf_counter() - t0) / reps
        info = r.info
        rows.append({"tol": tol, "ms": t * 1e3, "N": info["N"], "products": info["products"],
                     "density": info["nnz"] / n / n, "fma": info["fma"],
                     "dense_ms": info["products"] * t_gemm * 1e3})
    return {"workload": "banded_n65536_hbw5 exp", "dense_dgemm_s_projected": t_gemm, "rows": rows}


def measure_square(args, Z, flush):
    """cos and sinh on the headline workload, directly and with the W = Z^2
    substitution (PSF_Z_SQUARE): event-timed evaluations with L2 flushed
    before each, plan sizes, and the 1-norm distance between the two
    results (each is within tol of f(Z), so at most 2 tol apart)."""
    import numpy as np
    import scipy.sparse as sp
    import torch
    import paper_2208_05683_gb300 as psf
    import synthetic as syn
    from paper_2208_05683_gb300 import _abi
    L = psf.lib()
    stream = torch.cuda.current_stream()
    out = {}
    for kind in ("cos", "sinh"):
        row, mats = {}, {}
        # square_q2: the same with the PS block size q = 2 in W (s override)
        for mode, opts in (("direct", {}), ("square", {"square": True}), ("square_q2", {"square": True, "s": 2})):
            s = psf.Series(syn.coeffs(kind), TOL, kernel=args.kernel, **opts)
            lat = []
            for it in range(args.warmup + 2 * args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h = s.eval_handle(Z, stream)
                e1.record(stream)
                e1.synchronize()
                _abi.check(L.psf_result_destroy(h))
                if it >= args.warmup:
                    lat.append(e0.elapsed_time(e1))
            r = s.eval(Z)
            info = r.info
            rp, col, val = r.csr.to_host()
            mats[mode] = sp.csr_matrix((val, col, rp), shape=(Z.n, Z.n))
            row[mode] = {"p50_ms": statistics.median(lat), "evals_per_s": len(lat) / (sum(lat) / 1e3),
                         "N": info["N"], "q": info["q"], "b": info["b"], "products": info["products"],
                         "nnz": info["nnz"], "fma": info["fma"]}
        row["diff_1norm"] = float(abs(mats["direct"] - mats["square"]).sum(axis=0).max())
        row["diff_1norm_q2"] = float(abs(mats["direct"] - mats["square_q2"]).sum(axis=0).max())
        row["speedup_p50"] = row["direct"]["p50_ms"] / row["square"]["p50_ms"]
        row["speedup_p50_q2"] = row["direct"]["p50_ms"] / row["square_q2"]["p50_ms"]
        out[kind] = row
    out["how"] = f"{WORKLOAD}, tol {TOL:g}; {2 * args.steps} evaluations per mode after {args.warmup} warm-up"
    return out


def run_e2(args):
    """The paper's second experiment (Sec. 4, Figs. 1-2) on this GPU: random
    1000 x 1000 banded matrices, lower = upper bandwidth w = 1..15, N(0, 1)
    entries, `--e2-seeds` matrices per w, exp and cos at eps_tol = 1e-14.
    Per w: mean time of filtered PS (PSSCF), unfiltered PS and a dense FP64
    reference on the same GPU (torch.linalg.matrix_exp; cos(Z) = Re exp(iZ)
    in complex128), standing in for MATLAB's expm/cosm; the results'
    densities (nnz / n^2); and the relative errors of Eq. (39) against the
    dense reference, in the Frobenius norm and the 1-norm.  Times are wall
    clock through the Python API (one evaluation per matrix, after one
    untimed evaluation at each w), synchronized on both sides."""
    import numpy as np
    import torch
    import paper_2208_05683_gb300 as psf
    import synthetic as syn
    torch.cuda.set_device(0)
    dev = "cuda:0"
    n, tol, seeds = 1000, 1e-14, args.e2_seeds

    def dense_of(csr):
        rp, col, val = (torch.as_tensor(np.asarray(x)).to(dev) for x in csr)
        rows = torch.repeat_interleave(torch.arange(n, device=dev), (rp[1:] - rp[:-1]).long())
        X = torch.zeros(n, n, dtype=torch.float64, device=dev)
        X[rows, col.long()] = val.double()
        return X

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t0) * 1e3

    def reference(kind, Zd):
        if kind == "exp":
            return torch.linalg.matrix_exp(Zd)
        return torch.linalg.matrix_exp(1j * Zd.to(torch.complex128)).real.contiguous()

    def errors(res, ref):
        X = dense_of(res.csr.to_host())
        D = X - ref
        fro = float(torch.linalg.norm(D) / torch.linalg.norm(ref))
        one = float(torch.linalg.matrix_norm(D, ord=1) / torch.linalg.matrix_norm(ref, ord=1))
        return fro, one

    rows = []
    for kind in ("exp", "cos"):
        a = syn.coeffs(kind)
        filt, unf = psf.Series(a, tol, dense_xover=1e300), psf.Series(a, tol, filtered=False, dense_xover=1e300)
        # every product step as dense tiles, and the automatic choice
        dns, auto = psf.Series(a, tol, dense_xover=0.0), psf.Series(a, tol)
        # cos also with the W = Z^2 substitution (PSF_Z_SQUARE)
        sq = psf.Series(a, tol, square=True) if kind == "cos" else None
        for w in range(1, 16):
            acc = {k: [] for k in ("psscf_ms", "ps_ms", "ref_ms", "dense_tiles_ms", "auto_ms",
                                   "psscf_density", "ps_density", "ref_density",
                                   "psscf_err_fro", "ps_err_fro", "psscf_err_1", "ps_err_1", "N",
                                   "square_ms", "square_err_fro", "square_density")}
            for seed in range(seeds):
                host = syn.banded_normal(n, w, 1000 * w + seed)
                Z = psf.DeviceCSR.from_host(*host, device=dev)
                Zd = dense_of(host)
                if seed == 0:  # untimed first evaluation at this bandwidth
                    filt.eval(Z), unf.eval(Z), reference(kind, Zd), dns.eval(Z), auto.eval(Z)
                    if sq is not None:
                        sq.eval(Z)
                rf, tf = timed(lambda: filt.eval(Z))
                acc["dense_tiles_ms"].append(timed(lambda: dns.eval(Z))[1])
                acc["auto_ms"].append(timed(lambda: auto.eval(Z))[1])
                ru, tu = timed(lambda: unf.eval(Z))
                ref, tr = timed(lambda: reference(kind, Zd))
                ef, eu = errors(rf, ref), errors(ru, ref)
                acc["psscf_ms"].append(tf)
                acc["ps_ms"].append(tu)
                acc["ref_ms"].append(tr)
                acc["psscf_density"].append(rf.info["nnz"] / n / n)
                acc["ps_density"].append(ru.info["nnz"] / n / n)
                acc["ref_density"].append(float((ref != 0).sum()) / n / n)
                acc["psscf_err_fro"].append(ef[0])
                acc["ps_err_fro"].append(eu[0])
                acc["psscf_err_1"].append(ef[1])
                acc["ps_err_1"].append(eu[1])
                acc["N"].append(rf.info["N"])
                if sq is not None:
                    rs, ts = timed(lambda: sq.eval(Z))
                    acc["square_ms"].append(ts)
                    acc["square_err_fro"].append(errors(rs, ref)[0])
                    acc["square_density"].append(rs.info["nnz"] / n / n)
            row = {"kind": kind, "w": w}
            row.update({k: float(np.mean(v)) for k, v in acc.items() if v})
            row["psscf_err_fro_max"] = float(np.max(acc["psscf_err_fro"]))
            rows.append(row)
            print(f"{kind} w={w:2d}: psscf {row['psscf_ms']:7.2f} ms  dense tiles {row['dense_tiles_ms']:7.2f} ms  "
                  f"auto {row['auto_ms']:7.2f} ms  ps {row['ps_ms']:7.2f} ms  "
                  f"dense {row['ref_ms']:7.2f} ms  density {row['psscf_density']:.3f} / {row['ps_density']:.3f}  "
                  f"err {row['psscf_err_fro']:.2e} / {row['ps_err_fro']:.2e}  "
                  f"square {row.get('square_ms', float('nan')):7.2f} ms", file=sys.stderr, flush=True)
    print(json.dumps({"experiment": "banded_normal n=1000, w=1..15, N(0,1), exp and cos, eps_tol=1e-14",
                      "seeds_per_w": seeds, "reference": "torch.linalg.matrix_exp float64 / complex128 on the GPU",
                      "timing": "wall clock per evaluation through the Python API, synchronized", "rows": rows}))


def run_dense_xover(args):
    """Where dense tiles beat the sparse kernel: one product step C = A B of
    random matrices (n = 1000, 2000, 4000; densities spread so that the
    algorithmic multiply-adds per n^3 run from about 1e-4 to 1), timed
    through psf_product_filter as the sparse kernel and as dense tiles (the
    library's event timing of the product launches, median of 3), and the
    multiply-adds per n^3 from which dense tiles are faster."""
    import ctypes
    import numpy as np
    import scipy.sparse as sp
    import torch
    import paper_2208_05683_gb300 as psf
    from paper_2208_05683_gb300 import _abi
    torch.cuda.set_device(0)
    L = psf.lib()
    old = psf.tune_get(_abi.PSF_TUNE_DENSE_XOVER)
    rows = []
    try:
        for n in (1000, 2000, 4000):
            for d in (0.003, 0.01, 0.03, 0.06, 0.1, 0.2, 0.35, 0.6, 1.0):
                rng = np.random.default_rng(int(1000 * d) + n)
                mats = []
                for _ in range(2):
                    m = sp.random(n, n, density=d, random_state=rng, format="csr",
                                  data_rvs=lambda k: rng.uniform(-1, 1, k))
                    m.sort_indices()
                    mats.append(psf.DeviceCSR.from_host(m.indptr.astype(np.int32), m.indices.astype(np.int32),
                                                         m.data.astype(np.float64), device="cuda:0"))
                t = {}
                for name, v in (("sparse", 1e300), ("dense", 0.0)):
                    psf.tune_set(_abi.PSF_TUNE_DENSE_XOVER, v)
                    psf.product_filter(mats[0], mats[1], [], 0.0)
                    ms = []
                    for _ in range(3):
                        _abi.check(L.psf_profile(1))
                        r = psf.product_filter(mats[0], mats[1], [], 0.0)
                        nl, pms, fma = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
                        _abi.check(L.psf_profile_read(ctypes.byref(nl), ctypes.byref(pms), ctypes.byref(fma), 1))
                        _abi.check(L.psf_profile(0))
                        ms.append(pms.value)
                    t[name] = statistics.median(ms)
                    fma_n = r.steps[0]["fma"]
                rho = fma_n / float(n) ** 3
                rows.append({"n": n, "density": d, "fma_per_n3": rho, "sparse_ms": t["sparse"], "dense_ms": t["dense"],
                             "sparse_tflops": 2 * fma_n / t["sparse"] / 1e9,
                             "dense_tflops_on_n3": 2 * float(n) ** 3 / t["dense"] / 1e9})
                print(f"n={n} d={d}: fma/n^3 {rho:.2e}  sparse {t['sparse']:.3f} ms  dense {t['dense']:.3f} ms",
                      file=sys.stderr, flush=True)
                del mats
    finally:
        psf.tune_set(_abi.PSF_TUNE_DENSE_XOVER, old)
    cross = {}
    for n in sorted({r["n"] for r in rows}):
        rs = sorted((r for r in rows if r["n"] == n), key=lambda r: r["fma_per_n3"])
        win = [r["fma_per_n3"] for r in rs if r["dense_ms"] <= r["sparse_ms"]]
        cross[n] = min(win) if win else None
    print(json.dumps({"experiment": "one product step, random A B, sparse kernel vs dense tiles",
                      "crossover_fma_per_n3": cross, "rows": rows}))


def ctypes_i64(fn) -> int:
    import ctypes
    v = ctypes.c_int64()
    fn(ctypes.byref(v))
    return v.value


def run_case(args):
    """One evaluation of one series on the workload, nothing else: the
    command the ncu captures under profiles/ run."""
    import torch
    import paper_2208_05683_gb300 as psf
    import synthetic as syn
    torch.cuda.set_device(0)
    rp, col, val = syn.workload(args.case)[0]
    Z = psf.DeviceCSR.from_host(rp, col, val, device="cuda:0")
    # a pool large enough that no phase is repeated: kernel launch order is fixed
    series = psf.Series(syn.coeffs(args.kind), TOL, pool_entries=200_000_000, kernel=args.kernel)
    for _ in range(args.repeat):  # later evaluations use the earlier ones' statistics
        res = series.eval(Z)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "kind": args.kind, "nnz": res.csr.nnz, "N": res.info["N"],
                      "fma": res.info["fma"], "step_fma": [s["fma"] for s in res.steps],
                      "step_kind": [s["kind"] for s in res.steps]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default=None, help="run one evaluation of this workload and exit")
    ap.add_argument("--kind", default="exp")
    ap.add_argument("--repeat", type=int, default=1, help="with --case: evaluations of the one series")
    ap.add_argument("--kernel", choices=["auto", "table", "bitmap"], default="auto",
                    help="slot map of the product kernel (auto: by products per row)")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)  # 80 evaluations: p50/p99 over >= 20, clocks sampled
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["psf", "reference"], default="psf")
    ap.add_argument("--no-dense", action="store_true", help="skip the dense FP64 PS baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default slot-map crossover")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-instance batched measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-estimate", action="store_true", help="skip the estimated-norms (PSF_Z_ESTIMATE) measurement")
    ap.add_argument("--no-square", action="store_true",
                    help="skip the cos/sinh measurement with the W = Z^2 substitution (PSF_Z_SQUARE)")
    ap.add_argument("--serving-requests", type=int, default=10000, help="requests of the serving measurement")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the tolerance sweep of the banded n = 65536 workload against dense PS")
    ap.add_argument("--dense-full", action="store_true",
                    help="also run dense FP64 PS at the workload's full size (n = 16384, about a minute)")
    ap.add_argument("--e2", action="store_true",
                    help="run the paper's banded N(0,1) experiment (n = 1000, w = 1..15) and exit")
    ap.add_argument("--e2-seeds", type=int, default=30, help="matrices per bandwidth in --e2")
    ap.add_argument("--fp64-peak", action="store_true",
                    help="run the library's FP64 rate probe with the clocks sampled, print one JSON line and exit")
    ap.add_argument("--dense-xover", action="store_true",
                    help="time one product step as the sparse kernel and as dense tiles over densities and exit")
    ap.add_argument("--size-sweep", action="store_true",
                    help="time the 2D Laplacian workload on grids 128..768 (product kernel rate per size) and exit")
    args = ap.parse_args()
    if args.fp64_peak:
        import ctypes
        import torch
        import paper_2208_05683_gb300 as psf
        torch.cuda.set_device(0)
        runs = [fp64_probe(psf.lib(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), 0) for _ in range(3)]
        print(json.dumps({"experiment": "psf_fp64_peak", "nominal_2070": FP64_PEAK_TFLOPS, "runs": runs}))
    elif args.dense_xover:
        run_dense_xover(args)
    elif args.size_sweep:
        run_size_sweep(args)
    elif args.e2:
        run_e2(args)
    elif args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_psf(args)


if __name__ == "__main__":
    main()
