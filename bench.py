#!/usr/bin/env python3
"""Benchmark of the lattice convolution-sum evaluator on one B300 (or N, one process each).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (headline): BCC quintic box spline (the 4 BCC directions twice) on a BCC lattice of
2 x 128^3 FP32 coefficients sampled from the closed-form Marschner-Lobb signal, 2^24 uniform random
queries in the lattice interior, value and gradient.  One step = one interp_eval_grad over the
2^24 queries (every step of the evaluation path: cell reduction, fold, piece selection, gather,
Horner with derivatives, store).  Inputs are resident in HBM before the timed region; the points
(201 MB) are larger than L2.  Extra forms (plain FP32 value path, adjoint) are timed the same way
and reported under "forms".

Under torchrun (N > 1) every rank evaluates its own 2^24 queries (independent queries: weak
scaling, no data-path collective); the step time is the max over ranks.

--impl reference times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload (a deliberately slow baseline, not the target).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import LATTICES, SPLINES, WORKLOADS, coefficients, interior_box, make_rng, uniform_points  # noqa: E402

WORKLOAD = "bcc_quintic_128"
METRIC = "evals/s (value+grad, FP32, <=2e-6 rel err)"
UNIT = "evals/s"
SM_COUNT = 148
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2032.0


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


def fp32_peak_tflops():
    # derived: SMs x FP32 lanes x 2 FLOP per FMA x max SM clock
    return SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def workload_description(wl):
    return (f"{wl.name}: BCC quintic box spline (8 directions), 2 x {wl.dims[0]}^3 FP32 coefficients "
            f"sampled from the Marschner-Lobb signal, {wl.queries} uniform random queries in the lattice "
            f"interior, value + gradient")


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def recorded_traffic(kernel: str):
    """DRAM bytes per launch from the last ncu capture (profiles/traffic.txt), or None when the
    library sources changed since that capture."""
    from paper_2102_08514_b300 import build as b
    digest = b.source_digest()[:16]
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 3 and parts[0] == kernel and parts[1] == digest:
                    return int(parts[2])
    except OSError:
        pass
    return None


# ----------------------------------------------------------------------------- our arm

def time_steps(torch, fn, steps, warmup, stream, barrier):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    per = [a.elapsed_time(b) for a, b in ev]
    return t0.elapsed_time(t1), per


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if world == 1:
            return x
        t = torch.tensor([x], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    from paper_2102_08514_b300.binding import Interpolator

    wl = WORKLOADS[WORKLOAD]
    sp = SPLINES[wl.spline]
    lat = LATTICES[sp.lattice]
    itp = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), wl.dims, "f32")
    c = coefficients(wl)
    itp.set_coeffs(torch.from_numpy(c).cuda())
    lo, hi = interior_box(wl.spline, wl.dims)
    n = wl.queries
    pts_h = uniform_points(make_rng(wl.seed + 1000 * rank, 0), n, lo, hi)
    pts = torch.from_numpy(pts_h).cuda()
    out = torch.empty(n, device="cuda")
    grad = torch.empty(n, 3, device="cuda")
    gout = torch.from_numpy(make_rng(wl.seed, 5).uniform(-1, 1, n).astype(np.float32)).cuda()
    dcoef = torch.zeros(itp.shape, device="cuda")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()

    def step():
        itp.eval_grad(pts, out, grad)

    with ClockSampler(torch.cuda.current_device()) as clk:
        total_ms, per = time_steps(torch, step, args.steps, args.warmup, stream, barrier)
    clocks = clk.summary()
    total_ms = max_over_ranks(total_ms)
    ms_step = total_ms / args.steps
    value = world * n / (ms_step * 1e-3)

    # forms: plain FP32 value path and the adjoint, same timing rules
    fw = max(args.warmup, 3)
    fsteps = max(3, min(args.steps, 10))
    _, per_v = time_steps(torch, lambda: itp.eval(pts, out), fsteps, fw, stream, barrier)
    _, per_a = time_steps(torch, lambda: itp.backward(pts, gout, dcoef), fsteps, fw, stream, barrier)
    ms_v = statistics.mean(per_v)
    ms_a = statistics.mean(per_a)

    # e2e: points from pinned host memory, eval_grad, results back to pinned host memory
    pts_pin = torch.from_numpy(pts_h).pin_memory()
    out_pin = torch.empty(n, pin_memory=True)
    grad_pin = torch.empty(n, 3, pin_memory=True)
    pts_d = torch.empty_like(pts)

    def e2e_step():
        pts_d.copy_(pts_pin, non_blocking=True)
        itp.eval_grad(pts_d, out, grad)
        out_pin.copy_(out, non_blocking=True)
        grad_pin.copy_(grad, non_blocking=True)

    e2e_ms, _ = time_steps(torch, e2e_step, max(3, min(args.steps, 10)), fw, stream, barrier)
    e2e_ms = max_over_ranks(e2e_ms) / max(3, min(args.steps, 10))

    info = itp.info
    flops_per_launch = 2.0 * info.fma_grad_per_query * n
    kern_ms = statistics.mean(per)
    achieved = flops_per_launch / (kern_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    traffic = recorded_traffic(f"k_eval<{wl.spline},f32,grad>")
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded; Marschner-Lobb samples, uniform random queries)",
        "config": {"workload": workload_description(wl), "queries_per_gpu": n, "coeffs": list(itp.shape),
                   "parallelism": f"replicas x{world} (independent queries)",
                   "l2": "inputs larger than L2 (points 201 MB per GPU); coefficients (20 MB padded) stay L2-resident"},
        "e2e": {"value": world * n / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": n * 3 * 4,
                "d2h_bytes_per_step": n * 4 * 4},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": f"k_eval<{wl.spline},f32,value+grad>",
                     "flops_per_query": 2.0 * info.fma_grad_per_query,
                     "peak_note": "FP32 FMA peak derived: 148 SMs x 128 lanes x 2 FLOP x 2032 MHz"},
        "forms": {
            "value_grad": {"evals_per_s": n / (kern_ms * 1e-3), "ms": kern_ms},
            "value": {"evals_per_s": n / (ms_v * 1e-3), "ms": ms_v,
                      "tflops": 2.0 * info.fma_value_per_query * n / (ms_v * 1e-3) / 1e12},
            "adjoint": {"evals_per_s": n / (ms_a * 1e-3), "ms": ms_a},
        },
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, pts_h, c, seconds=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- the oracle (CPU)

def _oracle_setup(wl):
    import oracle
    sp = SPLINES[wl.spline]
    lat = LATTICES[sp.lattice]
    xi = np.asarray(sp.xi)
    detl = abs(round(np.linalg.det(np.asarray(lat.L, dtype=float))))
    return oracle, oracle.Spline(xi, detl), lat


def cpu_baseline(wl, pts, c, seconds=15.0):
    """Time the FP64 oracle (as it stands) on the host cores on a bounded sample."""
    orc, spl, lat = _oracle_setup(wl)
    cores = os.cpu_count() or 1
    cd = c.astype(np.float64)
    # grow the sample until it takes about `seconds` (bounded), then report the last one
    m, off = 4 * cores, 0
    while True:
        sample = pts[off:off + m].astype(np.float64)
        t = time.perf_counter()
        orc.eval_sum(spl, lat.D, lat.cosets, cd, sample, grad=True, nthreads=cores)
        dt = time.perf_counter() - t
        off += m
        if dt >= 0.5 * seconds or off + 2 * m > len(pts):
            break
        m = int(min(len(pts) - off, m * max(2.0, min(8.0, seconds / max(dt, 1e-3)))))
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{m} of the {wl.queries} queries (value+grad, FP64, brute-force recurrence), {dt:.1f} s"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[WORKLOAD]
    orc, spl, lat = _oracle_setup(wl)
    cores = os.cpu_count() or 1
    c = coefficients(wl).astype(np.float64)
    lo, hi = interior_box(wl.spline, wl.dims)
    pts = uniform_points(make_rng(wl.seed, 0), 1 << 16, lo, hi).astype(np.float64)
    # size each step so the whole run takes a few minutes
    probe = pts[:cores * 2]
    t = time.perf_counter()
    orc.eval_sum(spl, lat.D, lat.cosets, c, probe, grad=True, nthreads=cores)
    rate = len(probe) / max(time.perf_counter() - t, 1e-6)
    per_step = int(max(cores, min(len(pts) // (args.steps + args.warmup + 1), rate * 120.0 / (args.steps + args.warmup))))
    off = len(probe)

    def step(i):
        sl = pts[off + (i * per_step) % (len(pts) - off - per_step):][:per_step]
        orc.eval_sum(spl, lat.D, lat.cosets, c, sl, grad=True, nthreads=cores)

    for i in range(args.warmup):
        step(i)
    t = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = time.perf_counter() - t
    value = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": workload_description(wl), "sample_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} queries per step of the {wl.queries}-query workload"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
