#!/usr/bin/env python
"""Benchmark of the direct FFT Poisson solve on GB300.

One step = one full solve (x forward, y forward, z forward + eigenvalue
divide + z backward, y backward, x backward) of the 1024^3 FP32 workload
(periodic x, y; staggered Neumann z; second-order finite-difference
eigenvalues; seeded smooth Gaussian random field + 1e-3 white noise).  The
field (4 GiB) is far larger than L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  `value` is grid points solved per second
over all ranks, device-timed with CUDA events on the solve stream with the
inputs resident in HBM; `e2e` is the same metric through
poisfft_solve_host (host buffers; H2D + solve + D2H inside the timed
region); `roofline` covers the launch with the largest share of the step
time, timed live with per-launch CUDA events recorded by the library on the
same stream; `cpu_baseline` is the FP64 oracle on a bounded sample of the
same workload on this machine's host cores; `cufft_comparison` times cuFFT
(through torch.fft, all axes periodic) on the same field for context.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--impl ours|reference] [--no-check]

Multi-GPU (torchrun): every rank solves its own replica of the workload (the
solve has no cross-GPU exchange in this build), the step time is the max over
ranks and `value` counts all ranks' points ("scaling": "weak").
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "3D solve grid-pts/s & HBM-roofline fraction at 256^3/1024^3; max err vs FP64"
UNIT = "grid-pts/s"
DEFAULT_WORKLOAD = "ppn_fd2_1024_f32"
BC_NAME = {0: "P", 1: "DR", 2: "DS", 3: "NR", 4: "NS"}

# DRAM traffic / algorithmic bytes of the five specialised sweeps, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) on the
# 512x512x1024 workload (profiles/traffic_fast_sweeps_512x512x1024.md).
# Valid only while the kernel sources hash to TRAFFIC_SRC_SHA256.
TRAFFIC_RATIO = {("x_sweep", "forward"): 0.993, ("strided_sweep", "forward"): 0.993,
                 ("strided_sweep", "fused"): 0.999, ("strided_sweep", "backward"): 0.999,
                 ("x_sweep", "backward"): 0.993}
TRAFFIC_SRC_SHA256 = "f95fe083269be99bf624b220a50bc0ea0069f58f1801a91593a9b9fae401c829"
TRAFFIC_SOURCES = ["fast_kernels.cuh", "fft_engine.cuh", "fast_f32.cu"]


def kernel_source_sha256():
    import hashlib

    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1409_8116_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(W.WORKLOADS) + sorted(W.BATCHES) + sorted(W.VC_PROBLEMS) + sorted(W.LEARNED))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-check", action="store_true", help="skip the FP64 error check of the solution")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer (e2e) measurement")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT comparison")
    ap.add_argument("--no-size256", action="store_true", help="skip the 256^3 line beside the 1024^3 one")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision (refined) and FP64 direct solves beside the FP32 one")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def reduce_max(x: float, world: int, device: str = "cpu") -> float:
    """Max of a per-rank scalar over all ranks (the step time of the slowest
    rank); identity for one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(points_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job grid points per second: every rank solves its own replica."""
    return world * points_per_rank * steps / seconds


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_sample_oracle(spec, budget_s=12.0):
    """Time the FP64 oracle (dense Table 1 matrices) on the largest cubic
    sample of the workload's BC set that fits the time budget."""
    from oracle import poisson as O

    bcs, Ls, approx = spec["bcs"], spec["Ls"], spec["approx"]
    n = 32
    best = None
    while True:
        g = W.normal((n, n, n), 99, dtype=np.float64)
        t0 = time.perf_counter()
        O.solve(g, bcs, Ls, approx)
        dt = time.perf_counter() - t0
        best = (n, dt)
        if dt > budget_s / 8 or n >= 256:
            break
        n *= 2
    n, dt = best
    return {"value": n ** 3 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 oracle (dense Table-1 matrices, numpy/BLAS) on a {n}^3 grid with the workload's "
                      f"BCs {tuple(BC_NAME[b] for b in bcs)} and eigenvalues; {dt:.2f} s per solve"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import poisson as O

    spec = W.WORKLOADS[args.workload]
    bcs, Ls, approx = spec["bcs"], spec["Ls"], spec["approx"]
    # bounded sample of the workload: a cubic sub-grid sized for ~10 s per step
    n = 64
    g = W.normal((n, n, n), 5, dtype=np.float64)
    t0 = time.perf_counter()
    O.solve(g, bcs, Ls, approx)
    dt = time.perf_counter() - t0
    while dt < 1.5 and n < 256:
        n *= 2
        g = W.normal((n, n, n), 5, dtype=np.float64)
        t0 = time.perf_counter()
        O.solve(g, bcs, Ls, approx)
        dt = time.perf_counter() - t0
    for _ in range(args.warmup):
        O.solve(g, bcs, Ls, approx)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.solve(g, bcs, Ls, approx)
    total = time.perf_counter() - t0
    value = n ** 3 * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, spec),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"FP64 oracle (dense Table-1 matrices) on a {n}^3 sub-grid with the workload's "
                                   f"BCs and eigenvalues, per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cufft_comparison(g, warmup, steps):
    """The same field through cuFFT (torch.fft): 3D R2C, a pointwise multiply
    by a precomputed real factor (the divide), 3D C2R.  cuFFT has no DCT, so
    every axis is treated as periodic: the same class of work as the
    product's solve, not the same boundary conditions.  Device-timed with
    CUDA events; None when the field does not fit beside cuFFT's workspace."""
    import torch

    try:
        nz, ny, nx = g.shape
        fac = torch.rand((nz, ny, nx // 2 + 1), device=g.device, dtype=torch.float32)
        out = None
        for _ in range(max(1, warmup)):
            out = torch.fft.irfftn(torch.fft.rfftn(g) * fac, s=(nz, ny, nx))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            out = torch.fft.irfftn(torch.fft.rfftn(g) * fac, s=(nz, ny, nx))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        del out, fac
        torch.cuda.empty_cache()
        return {"ms_per_solve": ms, "points_per_s": nx * ny * nz / (ms / 1e3), "steps": steps,
                "what": "torch.fft (cuFFT) rfftn, multiply by a real factor, irfftn on the same FP32 field; "
                        "all axes periodic (cuFFT has no DCT)"}
    except RuntimeError as exc:  # out of memory next to the plan's buffers
        torch.cuda.empty_cache()
        return {"unavailable": str(exc).splitlines()[0][:200]}


def plan_singular(bcs):
    """Every axis periodic or Neumann: the solve removes the zero mode."""
    return all(b in (0, 3, 4) for b in bcs)


def workload_config(name, spec):
    nx, ny, nz = spec["n"]
    return {"workload": name, "n": [nx, ny, nz], "bcs": [BC_NAME[b] for b in spec["bcs"]],
            "approx": "spectral" if spec["approx"] == 0 else "fd2", "L": list(spec["Ls"]),
            "l2": "inputs larger than L2 (no flush needed)" if nx * ny * nz * 4 > 129e6 else "inputs smaller than L2, not flushed (not a headline workload)"}


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1409_8116_gb300 import binding as pb

    spec = W.WORKLOADS[args.workload]
    nx, ny, nz = spec["n"]
    npts = nx * ny * nz
    f64 = spec["dtype"] == "f64"
    tdt = torch.float64 if f64 else torch.float32
    esize = 8 if f64 else 4

    g_host = W.make_input(spec)
    plan = pb.Plan(spec["n"], spec["Ls"], spec["bcs"], spec["approx"], pb.F64 if f64 else pb.F32)
    launches = plan.launches()
    stream = torch.cuda.Stream()
    g = torch.from_numpy(g_host).to("cuda")
    phi = torch.empty_like(g)
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.solve(phi, g, stream)
    stream.synchronize()
    assert plan.check(stream) == pb.OK

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    # ---- timed region: K solves, per-launch events recorded by the library
    plan.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    e0.record(stream)
    for _ in range(args.steps):
        plan.solve(phi, g, stream)
    e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    plan.profile(False)
    ms_total = e0.elapsed_time(e1)
    per_launch_ms, nsolves = plan.profile_read()
    assert plan.check(stream) == pb.OK
    ms_max = reduce_max(ms_total, world, "cuda")
    value = throughput(npts, args.steps, world, ms_max / 1e3)

    # dominant launch: largest share of the step time
    shares = [t / sum(per_launch_ms) for t in per_launch_ms]
    dom = int(np.argmax(per_launch_ms))
    dom_ms = per_launch_ms[dom] / nsolves
    peak, peak_kind = load_peaks()
    achieved = launches[dom]["bytes"] / (dom_ms / 1e3) / 1e9
    traffic_valid = kernel_source_sha256() == TRAFFIC_SRC_SHA256

    def launch_traffic(i):
        key = (launches[i]["kernel"], launches[i]["mode"])
        return TRAFFIC_RATIO[key] * launches[i]["bytes"] if traffic_valid and key in TRAFFIC_RATIO else None

    traffic = launch_traffic(dom)
    per_launch = [dict(launches[i], ms=per_launch_ms[i] / nsolves, share=shares[i],
                       gbs=launches[i]["bytes"] / (per_launch_ms[i] / nsolves / 1e3) / 1e9,
                       frac=launches[i]["bytes"] / (per_launch_ms[i] / nsolves / 1e3) / 1e9 / peak,
                       traffic=launch_traffic(i))
                  for i in range(len(launches))]
    step_bytes = sum(l["bytes"] for l in launches)

    # ---- end to end through the host-buffer entry point
    e2e_value = e2e_same = e2e_sync = None
    if not args.no_e2e:
        gh = torch.from_numpy(g_host).pin_memory()
        ph = torch.empty_like(gh).pin_memory()
        e2e_steps = max(1, min(args.steps, 10))
        # K solves from and to host buffers through poisfft_solve_host_async
        # (every step copies its g in and its phi out inside the timed region;
        # consecutive steps overlap one step's result copy with the next input)
        for _ in range(max(1, args.warmup)):
            plan.solve_host_async(ph, gh, stream)
        assert plan.check(stream) == pb.OK
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            plan.solve_host_async(ph, gh, stream)
        assert plan.check(stream) == pb.OK  # waits for the last result copy too
        t_e2e = reduce_max(time.perf_counter() - t0, world, "cuda")
        e2e_value = throughput(npts, e2e_steps, world, t_e2e)
        # the synchronous call (one solve at a time), for comparison
        plan.solve_host(ph, gh, stream)
        t0 = time.perf_counter()
        for _ in range(min(e2e_steps, 5)):
            plan.solve_host(ph, gh, stream)
        e2e_sync = throughput(npts, min(e2e_steps, 5), world, reduce_max(time.perf_counter() - t0, world, "cuda"))
        # the host-buffer solve must give the device-resident result
        stride = max(1, npts // 100003)
        e2e_same = bool(torch.equal(ph.view(-1)[::stride], phi.cpu().view(-1)[::stride]))
        del gh, ph

    # ---- library comparison (not part of the product): cuFFT through torch.fft
    cufft = None
    if rank == 0 and not args.no_cufft:
        cufft = cufft_comparison(g, args.warmup, min(args.steps, 10))

    # ---- accuracy against the FP64 oracle (not timed)
    err = None
    if not args.no_check and rank == 0:
        from oracle import poisson as O

        ref = O.solve(g_host.astype(np.float64), spec["bcs"], spec["Ls"], spec["approx"],
                      method="dense" if npts <= 64 ** 3 else "fft")
        t_chk = time.perf_counter()
        err = O.rel_max_error(phi.cpu().numpy().astype(np.float64), ref)
        print(f"# FP64 check {time.perf_counter() - t_chk:.1f} s", file=sys.stderr)

    # ---- mixed-precision form next to the plain FP32 solve (not the headline)
    mixed = None
    if rank == 0 and not args.no_mixed and not f64 and spec["approx"] == pb.FD2:
        mixed = mixed_form(pb, plan, spec, g_host, ref if err is not None else None, stream, args)
    tcf = None
    if rank == 0 and not args.no_mixed and not f64:
        tcf = tensor_core_form(pb, spec, g, ref if err is not None else None, stream, args)
    if err is not None:
        del ref
    zero_mode = None
    if rank == 0 and plan_singular(spec["bcs"]):
        zero_mode = {"mean_fp64_gpu": plan.zero_mode_mean(g, stream)}
        if not args.no_check:
            from oracle import poisson as O

            zero_mode["mean_fp64_oracle"] = O.weighted_mean(g_host.astype(np.float64), spec["bcs"])

    cpu = cpu_fft = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample_oracle(spec)
        cpu_fft = cpu_fft_baseline(spec)
    size256 = None
    if rank == 0 and args.workload == DEFAULT_WORKLOAD and not args.no_size256:
        size256 = size_256_line(pb, args, peak)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if f64 else "f32", "data": "synthetic",
            "config": workload_config(args.workload, spec),
            "max_rel_err_vs_fp64": err, "zero_mode": zero_mode, "cufft_comparison": cufft,
            "mixed_precision": mixed, "bf16x3_tensor_core": tcf,
            "hbm_frac_step": step_bytes * args.steps / (ms_max / 1e3) / 1e9 / peak,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": f"{launches[dom]['kernel']} ({launches[dom]['mode']}, axis {launches[dom]['axis']})",
                         "peak_source": f"{peak_kind} hbm_gbs"},
            "launches": per_launch,
            "cpu_baseline": cpu, "cpu_fft_baseline": cpu_fft, "size_256": size256,
            "e2e": None if e2e_value is None else {
                "value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": npts * esize,
                "d2h_bytes_per_step": npts * esize,
                "path": "poisfft_solve_host_async: pinned host buffers, one copy each way through two alternating "
                        "device staging pairs, K calls then poisfft_check (waits for the last result copy)",
                "synchronous_call_value": e2e_sync, "equals_device_result": e2e_same},
            "gpu_launches": len(launches) * args.steps,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def mixed_form(pb, plan, spec, g_host, ref, stream, args):
    """FP64 data solved by FP32 FFT solves refined with FP64 residuals of the
    FD2 operator (poisfft_solve_refined), timed next to the FP64 direct solve
    of the same problem; errors against the FP64 oracle's solution."""
    import torch

    g64 = torch.from_numpy(g_host.astype(np.float64)).to("cuda")
    phi64 = torch.empty_like(g64)
    ref_d = torch.from_numpy(ref).to("cuda") if ref is not None else None
    ref_max = float(ref_d.abs().max()) if ref_d is not None else None

    def rel_err(x):
        return None if ref_d is None else float((x - ref_d).abs().max()) / ref_max

    def timed(fn, steps):
        for _ in range(max(1, min(args.warmup, 2))):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / steps

    out = {"what": "float64 g and phi; FP32 FFT solves of this plan refined with FP64 residuals of the FD2 "
                   "operator (poisfft_solve_refined), against the FP64 direct solve (FP64 plan) on the same GPU"}
    steps = max(1, min(args.steps, 5))
    for k in (1, 2):
        ms = timed(lambda: plan.solve_refined(phi64, g64, k, stream), steps)
        out[f"refinements_{k}"] = {"ms_per_solve": ms, "max_rel_err_vs_fp64": rel_err(phi64)}
    plan64 = pb.Plan(spec["n"], spec["Ls"], spec["bcs"], spec["approx"], pb.F64)
    ms64 = timed(lambda: plan64.solve(phi64, g64, stream), max(1, min(args.steps, 2)))
    assert plan64.check(stream) == pb.OK
    out["fp64_direct"] = {"ms_per_solve": ms64, "max_rel_err_vs_fp64": rel_err(phi64)}
    plan64.close()
    del g64, phi64, ref_d
    torch.cuda.empty_cache()
    return out


def cpu_fft_baseline(spec, n=256):
    """The paper's method on the host cores: the FP64 oracle's scipy.fft
    realisation of the Table 2 transforms (workers = every core), standing
    in for the paper's FFTW build, on an n^3 sample with the workload's BCs."""
    from oracle import poisson as O

    g = W.normal((n, n, n), 98, dtype=np.float64)
    O.solve(g, spec["bcs"], spec["Ls"], spec["approx"], method="fft")  # warm-up (plans, threads)
    t0 = time.perf_counter()
    reps = 2
    for _ in range(reps):
        O.solve(g, spec["bcs"], spec["Ls"], spec["approx"], method="fft")
    dt = (time.perf_counter() - t0) / reps
    return {"value": n ** 3 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "fft",
            "sample": f"FP64 scipy.fft (pocketfft, workers = all cores) solve of a {n}^3 grid with the workload's "
                      f"BCs {tuple(BC_NAME[b] for b in spec['bcs'])}; {dt:.2f} s per solve"}


def size_256_line(pb, args, peak):
    """The metric's second size, 256^3 (P, DS, NS), FD2, FP32: the field
    (64 MiB) is smaller than L2, so a 512 MiB buffer is written between
    timed solves; each solve is timed alone with CUDA events on its stream."""
    import torch

    name = "mixed_fd2_256_f32"
    spec = W.WORKLOADS[name]
    g_host = W.make_input(spec)
    npts = int(np.prod(spec["n"]))
    plan = pb.Plan(spec["n"], spec["Ls"], spec["bcs"], spec["approx"], pb.F32)
    launches = plan.launches()
    stream = torch.cuda.Stream()
    g = torch.from_numpy(g_host).to("cuda")
    phi = torch.empty_like(g)
    flush = torch.empty(128 << 20, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            plan.solve(phi, g, stream)
    steps = max(5, min(args.steps, 50))
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    plan.profile(True)
    with torch.cuda.stream(stream):
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            plan.solve(phi, g, stream)
            e1.record(stream)
    stream.synchronize()
    plan.profile(False)
    per, ns = plan.profile_read()
    assert plan.check(stream) == pb.OK
    ms = sum(e0.elapsed_time(e1) for e0, e1 in evs) / steps
    dom = int(np.argmax(per))
    dom_ms = per[dom] / ns
    achieved = launches[dom]["bytes"] / (dom_ms / 1e3) / 1e9
    step_bytes = sum(l["bytes"] for l in launches)
    err = None
    if not args.no_check:
        from oracle import poisson as O

        ref = O.solve(g_host.astype(np.float64), spec["bcs"], spec["Ls"], spec["approx"], method="fft")
        err = O.rel_max_error(phi.cpu().numpy().astype(np.float64), ref)
    out = {"config": workload_config(name, spec), "value": npts / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "steps": steps, "l2": "512 MiB written between timed solves (field smaller than L2)",
           "hbm_frac_step": step_bytes / (ms / 1e3) / 1e9 / peak,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                        "kernel": f"{launches[dom]['kernel']} ({launches[dom]['mode']}, axis {launches[dom]['axis']})"},
           "launches": [dict(kernel=l["kernel"], mode=l["mode"], axis=l["axis"], ms=per[i] / ns)
                        for i, l in enumerate(launches)],
           "max_rel_err_vs_fp64": err}
    if not args.no_cufft:
        out["cufft_comparison"] = cufft_comparison(g, args.warmup, min(args.steps, 10))
    if not args.no_cpu_baseline:
        out["cpu_fft_baseline"] = cpu_fft_baseline(spec)
    plan.close()
    del g, phi, flush
    torch.cuda.empty_cache()
    return out


def tensor_core_form(pb, spec, g, ref, stream, args):
    """The same FP32 field solved by a POISFFT_BF16X3 plan: the DFT blocks of
    the 1024-point strided axes as split-BF16 tensor-core GEMMs (tcgen05,
    FP32 accumulation); time per solve, per-launch times and the error
    against the FP64 oracle.  None when the plan has no such axis."""
    import torch

    try:
        plan = pb.Plan(spec["n"], spec["Ls"], spec["bcs"], spec["approx"], pb.BF16X3)
    except pb.PoisFFTError as e:
        return {"unavailable": str(e)}
    phi = torch.empty_like(g)
    for _ in range(max(1, min(args.warmup, 3))):
        plan.solve(phi, g, stream)
    stream.synchronize()
    steps = max(1, min(args.steps, 10))
    plan.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.solve(phi, g, stream)
    e1.record(stream)
    stream.synchronize()
    plan.profile(False)
    per, ns = plan.profile_read()
    assert plan.check(stream) == pb.OK
    launches = plan.launches()
    out = {"what": "POISFFT_BF16X3 plan: radix-32 DFT blocks of the 1024-point strided axes as tcgen05 GEMMs "
                   "with hi/lo bfloat16 operands (three products, FP32 accumulation); other sweeps FP32",
           "ms_per_solve": e0.elapsed_time(e1) / steps,
           "launches": [dict(kernel=l["kernel"], mode=l["mode"], axis=l["axis"], ms=per[i] / ns)
                        for i, l in enumerate(launches)],
           "max_rel_err_vs_fp64": None}
    if ref is not None:
        ref_d = torch.from_numpy(ref).to("cuda")
        out["max_rel_err_vs_fp64"] = float((phi.double() - ref_d).abs().max()) / float(ref_d.abs().max())
        del ref_d
    plan.close()
    del phi
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    """Batched workload: every step solves all problems once through the
    batch's CUDA graph.  Also times the plain form (the same problems one
    after another, no graph) for the speedup."""
    import torch

    from paper_1409_8116_gb300 import binding as pb

    spec = W.BATCHES[args.workload]
    probs = W.batch_problems(spec["count"], spec["seed"])
    npts = sum(int(np.prod(p["n"])) for p in probs)
    t0 = time.perf_counter()
    batch = pb.Batch([(p["n"], p["Ls"], p["bcs"]) for p in probs], spec["approx"], pb.F32)
    t_create = time.perf_counter() - t0
    gs = [torch.from_numpy(W.normal(tuple(reversed(p["n"])), p["gseed"], dtype=np.float32)).cuda() for p in probs]
    phis = [torch.empty_like(x) for x in gs]
    stream = torch.cuda.Stream()
    t0 = time.perf_counter()
    chosen, tune_ms = batch.autotune(phis, gs, stream)
    t_tune = time.perf_counter() - t0
    for _ in range(args.warmup):
        batch.solve(phis, gs, stream)
    stream.synchronize()
    assert batch.check(stream) == pb.OK

    def timed(fn, steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn(phis, gs, stream)
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1)

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ms_graph = timed(batch.solve, args.steps)
    clocks = sampler.stop()
    for _ in range(args.warmup):
        batch.solve_sequential(phis, gs, stream)
    ms_plain = timed(batch.solve_sequential, args.steps)
    # the plain form at its best: every plan's tiles tuned alone
    plain_by_config = {}
    for cand, cname in enumerate(pb.Batch.TUNE_CANDIDATES):
        batch.select(cand)
        for _ in range(max(1, args.warmup)):
            batch.solve_sequential(phis, gs, stream)
        plain_by_config[cname] = timed(batch.solve_sequential, args.steps) / args.steps
    batch.select(chosen)
    ms_plain_best = min(plain_by_config.values()) * args.steps
    # one persistent launch per sweep phase over all problems
    persistent = None
    try:
        for _ in range(max(1, args.warmup)):
            batch.solve_persistent(phis, gs, stream)
        ms_pers = timed(batch.solve_persistent, args.steps)
        persistent = {"ms_per_step": ms_pers / args.steps, "value": throughput(npts, args.steps, 1, ms_pers / 1e3)}
    except pb.PoisFFTError as e:
        persistent = {"unavailable": str(e)}
    assert batch.check(stream) == pb.OK
    value = throughput(npts, args.steps, 1, ms_graph / 1e3)
    err = None
    if not args.no_check:
        from oracle import poisson as O

        batch.solve(phis, gs, stream)
        stream.synchronize()
        worst = 0.0
        for p, g, phi in zip(probs, gs, phis):  # every problem of the batch
            ref = O.solve(g.cpu().numpy().astype(np.float64), p["bcs"], p["Ls"], spec["approx"], method="fft")
            worst = max(worst, O.rel_max_error(phi.cpu().numpy(), ref))
        err = worst
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import poisson as O

        sample = sorted(probs, key=lambda p: int(np.prod(p["n"])))[:32]
        t0 = time.perf_counter()
        for p in sample:
            O.solve(W.normal(tuple(reversed(p["n"])), p["gseed"], dtype=np.float64), p["bcs"], p["Ls"], spec["approx"])
        dt = time.perf_counter() - t0
        cpu = {"value": sum(int(np.prod(p["n"])) for p in sample) / dt, "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle", "sample": "FP64 oracle (dense Table-1 matrices) on the 32 smallest problems of the "
                                           f"batch ({dt:.1f} s)"}
    peak, peak_kind = load_peaks()
    info = batch.info()
    achieved = info["bytes"] / (ms_graph / args.steps / 1e3) / 1e9
    # end to end: pinned host inputs copied in, one graph replay, solutions
    # copied back, every step
    e2e = None
    if not args.no_e2e:
        gh = [x.cpu().pin_memory() for x in gs]
        ph = [torch.empty_like(x).pin_memory() for x in gh]
        gd2 = [torch.empty_like(x) for x in gs]
        pd2 = [torch.empty_like(x) for x in gs]

        def e2e_step():
            with torch.cuda.stream(stream):
                for d, h in zip(gd2, gh):
                    d.copy_(h, non_blocking=True)
                batch.solve(pd2, gd2, stream)
                for h, d in zip(ph, pd2):
                    h.copy_(d, non_blocking=True)
            stream.synchronize()

        e2e_step()
        e2e_steps = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        t_e2e = time.perf_counter() - t0
        nbytes = sum(x.numel() * 4 for x in gs)
        e2e = {"value": npts * e2e_steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes,
               "path": "pinned host buffers, one copy per problem each way, batch graph replay in between"}
        del gh, ph, gd2, pd2
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_graph / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": args.workload, "problems": len(probs), "points": npts,
                   "dims2": sum(p["dims"] == 2 for p in probs), "approx": "fd2",
                   "l2": "inputs larger than L2 (2.7 GB over the batch)"},
        "plain_ms_per_step": ms_plain / args.steps, "plain_ms_per_step_by_config": plain_by_config,
        "speedup_vs_best_plain": ms_plain_best / ms_graph, "speedup_vs_plain_same_tiles": ms_plain / ms_graph,
        "persistent_phases": persistent,
        "create_s": t_create, "max_rel_err_vs_fp64": err, "checked_problems": None if err is None else len(probs),
        "autotune": {"kept": pb.Batch.TUNE_CANDIDATES[chosen],
                     "ms_per_replay": dict(zip(pb.Batch.TUNE_CANDIDATES, tune_ms)), "seconds": t_tune},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "bytes_per_step": info["bytes"],
                     "kernel": "whole batch graph: algorithmic bytes of every launch of every problem / replay time",
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": info["launches"] * args.steps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    batch.close()
    return 0


PCG_METRIC = "variable-coefficient PCG: cell-iterations/s (FFT preconditioner), time to tolerance"
PCG_UNIT = "cell-iterations/s"
# Algorithmic bytes per cell and iteration of the mixed-precision iteration:
# operator 20 (p, three FP32 face coefficients, q), update 24 (e and r read
# and written, p, q), preconditioner inner products 12 (r and two
# preconditioner outputs), direction 12 (output, p read and written), and
# the FP32 Poisson solve as five sweeps that read and write 4 B each.
PCG_BYTES_OWN = 68
PCG_BYTES_POISSON = 40


def run_pcg(args):
    """Variable-coefficient workload: one step = one PCG solve from phi = 0
    to the workload's tolerance (mixed precision: FP32 iterations, FP64
    reliable updates; the FP64 iteration is timed beside it).  `value`
    counts cells x iterations per second; the solve time and the iteration
    count are reported beside it."""
    import torch

    from paper_1409_8116_gb300 import binding as pb

    spec = W.VC_PROBLEMS[args.workload]
    n = spec["n"]
    shape = tuple(reversed(n))
    npts = int(np.prod(n))
    a_host = W.lognormal_coefficient(shape, spec["seed"], spec["contrast"])
    g_host = W.normal(shape, spec["seed"] + 1)
    stream = torch.cuda.Stream()
    a = torch.from_numpy(a_host).cuda()
    g = torch.from_numpy(g_host).cuda()
    phi = torch.zeros_like(g)
    solver = pb.PCG(n, spec["Ls"], a)
    torch.cuda.synchronize()

    def timed(precision, steps, warmup):
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                phi.zero_()
                solver.solve(phi, g, spec["tol"], 1000, stream, precision)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            iters = []
            e0.record(stream)
            for _ in range(steps):
                phi.zero_()
                its, rel = solver.solve(phi, g, spec["tol"], 1000, stream, precision)
                iters.append(its)
            e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1), iters, rel, solver.stats()

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    ms, iters, rel, stats = timed(pb.PCG_MIXED, args.steps, args.warmup)
    clocks = sampler.stop()
    sol = phi.cpu().numpy()
    # kernel launches of one mixed solve: residual + check, one Poisson solve
    # (the preconditioner plan's sweeps) and two kernels per preconditioner
    # application, six kernels per loop iteration (one loop iteration per
    # application after the first), three closing kernels
    with pb.Plan(n, spec["Ls"], (W.DS, W.DS, W.DS), pb.FD2, pb.F32) as pplan:
        plan_launches = len(pplan.launches())
    npre = stats["preconditioner_solves"]
    launches_per_solve = 2 + npre * (plan_launches + 2) + (npre - 1) * 6 + 3

    e2e = None
    if not args.no_e2e:
        # end to end: g from pinned host memory, phi back to pinned host memory
        gh = torch.from_numpy(g_host).pin_memory()
        ph = torch.empty_like(gh).pin_memory()
        e2e_steps = max(1, min(args.steps, 5))
        e2e_it = 0
        with torch.cuda.stream(stream):
            for k in range(e2e_steps + 1):
                if k == 1:
                    stream.synchronize()
                    t0 = time.perf_counter()
                g.copy_(gh, non_blocking=True)
                phi.zero_()
                its, _ = solver.solve(phi, g, spec["tol"], 1000, stream, pb.PCG_MIXED)
                ph.copy_(phi, non_blocking=True)
                if k > 0:
                    e2e_it += its
            stream.synchronize()
        t_e2e = time.perf_counter() - t0
        e2e = {"value": npts * e2e_it / t_e2e, "unit": PCG_UNIT, "ms_per_solve": t_e2e / e2e_steps * 1e3,
               "h2d_bytes_per_step": g.numel() * g.element_size(),
               "d2h_bytes_per_step": phi.numel() * phi.element_size(),
               "path": "g from pinned host memory, PCG solve (poisfft_pcg_solve), phi to pinned host memory"}
        del gh, ph
    ms64, iters64, rel64, _ = timed(pb.PCG_F64, max(1, min(args.steps, 3)), 1)
    total_it = sum(iters)
    value = npts * total_it / (ms / 1e3)
    true_rel = None
    if not args.no_check:
        from oracle import vc_operator as V

        true_rel = float(np.linalg.norm(g_host - V.apply_operator(sol, a_host.astype(np.float64), spec["Ls"]))
                         / np.linalg.norm(g_host))
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import vc_operator as V

        m = 96
        sa = W.lognormal_coefficient((m, m, m), spec["seed"], spec["contrast"]).astype(np.float64)
        sg = W.normal((m, m, m), spec["seed"] + 1)
        t0 = time.perf_counter()
        _, cit, _ = V.pcg(sg, sa, spec["Ls"], tol=spec["tol"], maxit=12)
        dt = time.perf_counter() - t0
        cpu = {"value": m ** 3 * cit / dt, "unit": PCG_UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 oracle PCG on {m}^3 cells of the same recipe, {cit} iterations ({dt:.1f} s)"}
    peak, peak_kind = load_peaks()
    ms_it = ms / total_it
    achieved = npts * (PCG_BYTES_OWN + PCG_BYTES_POISSON) / (ms_it / 1e3) / 1e9
    n64 = len(iters64)
    line = {
        "metric": PCG_METRIC, "value": value, "unit": PCG_UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 iterations + f64 reliable updates", "data": "synthetic",
        "config": {"workload": args.workload, "n": list(n), "contrast": spec["contrast"], "tol": spec["tol"],
                   "l2": "inputs larger than L2 (no flush needed)"},
        "iterations": iters[-1], "ms_per_iteration": ms_it, "relres": rel, "true_relres": true_rel,
        "fp64_true_residuals": stats["true_residuals"],
        "f64_iteration": {"ms_per_solve": ms64 / n64, "iterations": iters64[-1], "relres": rel64,
                          "ms_per_iteration": ms64 / sum(iters64)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "whole mixed PCG iteration (own kernels + FP32 Poisson solve)",
                     "bytes_per_cell_iteration": PCG_BYTES_OWN + PCG_BYTES_POISSON,
                     "peak_source": f"{peak_kind} hbm_gbs"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches_per_solve * args.steps, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    solver.close()
    return 0


def run_learned(args):
    """Learned form: train the spectral neural operator on pairs from the
    library's PCG (coarse grid), then time the PCG on the 256^3 problem from
    phi = 0 and from the learned guess (0, 1, 2 residual corrections), to the
    same relative residual.  One step = one solve including the network."""
    import torch

    from paper_1409_8116_gb300 import binding as pb
    from paper_1409_8116_gb300 import learned

    spec = W.LEARNED[args.workload]
    ev = W.VC_PROBLEMS[spec["eval"]]
    arch = spec["arch"]
    t0 = time.perf_counter()
    samples = W.learned_samples(spec["n_train"], spec["pairs"] + spec["holdout"], spec["seed"], spec["contrast"])
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    feats, targets, info = learned.generate_pairs(spec["n_train"], ev["Ls"], samples, tol=spec["pair_tol"])
    t_pairs = time.perf_counter() - t0
    theta, hist = learned.train((feats, targets), spec["n_train"], batch=spec["batch"], epochs=spec["epochs"],
                                lr=spec["lr"], seed=spec["seed"], holdout=spec["holdout"], **arch)
    del feats, targets
    torch.cuda.empty_cache()

    def solve_set(n, Ls, a, g, net, steps, warm):
        out = {}
        stream = torch.cuda.Stream()
        with pb.PCG(n, Ls, torch.from_numpy(a).cuda()) as pcg:
            gd = torch.from_numpy(g).cuda()
            phi = torch.zeros_like(gd)
            for mode in ("plain", "learned0", "learned1", "learned2"):
                corr = None if mode == "plain" else int(mode[-1])

                def one():
                    if corr is None:
                        phi.zero_()
                    else:
                        pcg.learned_guess(net, phi, gd, corrections=corr, stream=stream)
                    return pcg.solve(phi, gd, tol=ev["tol"], maxit=1000, stream=stream)

                with torch.cuda.stream(stream):
                    for _ in range(warm):
                        one()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(steps):
                        it, rel = one()
                    e1.record(stream)
                stream.synchronize()
                out[mode] = {"ms": e0.elapsed_time(e1) / steps, "iterations": it, "relres": rel}
        return out

    shape = tuple(reversed(ev["n"]))
    a = W.lognormal_coefficient(shape, ev["seed"], ev["contrast"])
    g = W.normal(shape, ev["seed"] + 1)
    net = learned.load_network(ev["n"], theta, **arch)
    # network inference alone (one forward on the 256^3 features)
    Nc = int(np.prod(ev["n"]))
    fin = torch.randn((3, Nc), device="cuda")
    yout = torch.empty(Nc, device="cuda")
    for _ in range(2):
        net.forward(yout, fin)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        net.forward(yout, fin)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 5
    C, Lyr = arch["channels"], arch["layers"]
    # algorithmic bytes per cell of one forward (FP32 activations): lifting
    # reads 3 features and writes C channels; per layer the sine analysis reads
    # C, the channel mixing reads C and writes C; the projection reads C, writes 1
    fwd_bytes = Nc * 4 * ((3 + C) + Lyr * 3 * C + (C + 1))
    del fin, yout
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    res = solve_set(ev["n"], ev["Ls"], a, g, net, args.steps, args.warmup)
    clocks = sampler.stop()
    best = min(("learned0", "learned1", "learned2"), key=lambda k: res[k]["ms"])

    e2e = None
    if not args.no_e2e:
        # the same ratio end to end: g from pinned host memory, phi back to it
        def e2e_ms(corr, steps=3):
            stream = torch.cuda.Stream()
            with pb.PCG(ev["n"], ev["Ls"], torch.from_numpy(a).cuda()) as pcg:
                gh = torch.from_numpy(g).pin_memory()
                ph = torch.empty_like(gh).pin_memory()
                gd = torch.empty(gh.shape, dtype=gh.dtype, device="cuda")
                phi = torch.zeros_like(gd)
                with torch.cuda.stream(stream):
                    for k in range(steps + 1):
                        if k == 1:
                            stream.synchronize()
                            t0 = time.perf_counter()
                        gd.copy_(gh, non_blocking=True)
                        if corr is None:
                            phi.zero_()
                        else:
                            pcg.learned_guess(net, phi, gd, corrections=corr, stream=stream)
                        pcg.solve(phi, gd, tol=ev["tol"], maxit=1000, stream=stream)
                        ph.copy_(phi, non_blocking=True)
                    stream.synchronize()
                return (time.perf_counter() - t0) / steps * 1e3

        plain_ms, learned_ms = e2e_ms(None), e2e_ms(int(best[-1]))
        e2e = {"value": plain_ms / learned_ms, "unit": "x (speedup, >1 = learned faster)",
               "plain_ms": plain_ms, "learned_ms": learned_ms,
               "h2d_bytes_per_step": g.size * 8, "d2h_bytes_per_step": g.size * 8,
               "path": "g from pinned host memory, PCG solve from zero or from the learned guess, phi to pinned host memory"}
    net.close()
    net64 = learned.load_network(spec["n_train"], theta, **arch)
    held = []
    for a_h, g_h in samples[spec["pairs"]:spec["pairs"] + 4]:
        r = solve_set(spec["n_train"], ev["Ls"], a_h, g_h, net64, 2, 1)
        held.append({k: v["iterations"] for k, v in r.items()})
    net64.close()
    line = {
        "metric": "learned PCG: time to 1e-8 relative residual, plain FFT-preconditioned PCG / with the learned guess",
        "value": res["plain"]["ms"] / res[best]["ms"], "unit": "x (speedup, >1 = learned faster)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res[best]["ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "network bf16 weights / f32 activations; PCG f32 iterations + f64 reliable updates",
        "data": "synthetic", "config": {"workload": args.workload, "eval": spec["eval"], "n": list(ev["n"]),
                                        "n_train": list(spec["n_train"]), "pairs": spec["pairs"], **arch,
                                        "epochs": spec["epochs"], "batch": spec["batch"]},
        "eval_256": res, "best": best, "heldout_train_grid_iterations": held,
        "train": {"host_gen_s": t_gen, "pairs_s": t_pairs, "train_s": hist["seconds"],
                  "loss_first_epoch": hist["train_loss"][0], "loss_last_epoch": hist["train_loss"][-1],
                  "holdout_loss": hist["holdout_loss"][-1] if hist["holdout_loss"] else None,
                  "pair_pcg_iterations_mean": float(np.mean(info["pcg_iterations"]))},
        "network_forward_ms": fwd_ms,
        "roofline": {"bound": "hbm", "achieved": fwd_bytes / (fwd_ms / 1e3) / 1e9, "peak": load_peaks()[0],
                     "unit": "GB/s", "frac": fwd_bytes / (fwd_ms / 1e3) / 1e9 / load_peaks()[0], "traffic": None,
                     "kernel": "network forward at 256^3 (all its kernels)",
                     "bytes_per_cell": fwd_bytes / Nc, "peak_source": f"{load_peaks()[1]} hbm_gbs"},
        "cpu_baseline": None, "e2e": e2e, "gpu_launches": None, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in W.BATCHES:
        return run_batch(args)
    if args.workload in W.VC_PROBLEMS:
        return run_pcg(args)
    if args.workload in W.LEARNED:
        return run_learned(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
