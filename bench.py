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
import dataclasses
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
# default timed form per workload (the headline is bcc_quintic_128: value + gradient)
DEFAULT_FORM = {"bcc_linear_16": "value", "bcc_quintic_128": "value_grad", "fcc_6dir_128": "value_grad",
                "cc_7dir_256": "value", "d4s_8dir_48": "value"}
UNIT = "evals/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def presort_applies(info, n: int) -> bool:
    """Whether an evaluation call of n queries takes the library's piece pre-sort: its default for
    this spline (interp_info_t.presort) at >= 2^16 queries, or INTERP_B300_PRESORT=0 / 1 (any
    spline whose evaluation runs the piece-binned kernels, interp_info_t.binned)."""
    env = os.environ.get("INTERP_B300_PRESORT")
    if env:
        return env[0] == "1" and bool(info.binned)
    return bool(info.presort) and n >= (1 << 16)


def adjoint_bins_apply(info, n: int) -> bool:
    """Whether interp_backward on n queries takes the binned adjoint with the handle's default
    options (the library's rule: 3-D spline with < 4 pieces and >= 24 lookups per query, and the
    contributions at least four times the sites of the bins' shared-memory boxes; bins of 8^3
    coset cells over the padded arrays, boxes of 8 + 2 halo + 2 sites per axis and coset), or
    INTERP_B300_ADJOINT_BINS=0 / 1."""
    if info.s != 3 or info.n_pieces >= 4 or info.D > 2:
        return False
    env = os.environ.get("INTERP_B300_ADJOINT_BINS")
    if env:
        return env[0] == "1"
    if info.lookups_per_query < 24:
        return False
    nbins = 1
    for a in range(3):
        pdims = -(-(info.dims[a] + 4 * info.halo) // 2) * 2
        nbins *= -(-pdims // 8)
    w = 8 + 2 * info.halo + 2
    return n * info.lookups_per_query >= 4.0 * nbins * info.n_cosets * w ** 3


def launches_per_step(form: str, n: int, presort: bool, adjoint_bins: bool = False) -> int:
    """This library's kernels in one step: the evaluation kernel (value forms), or the adjoint
    kernel and the unpadding add (adjoint); the binned adjoint adds its count, scan and scatter
    kernels; with the pre-sort, per chunk of 2^22 queries the piece classifier, count, scan and
    scatter kernels before the evaluation (adjoint) kernel, and the un-permute after it (value
    forms)."""
    chunks = -(-n // (1 << 22))
    if form == "adjoint":
        if adjoint_bins:
            return 5
        return (5 * chunks if presort else 1) + 1
    return 6 * chunks if presort else 1


_PEAKS = {}


def measured_peaks(torch):
    """The rooflines' denominators, measured on this GPU in this run by the microbenchmarks of
    paper_2102_08514_b300/peaks.py (FP32 FMA rate, random-gather sector rate, L2 atomic rate, L2
    read bandwidth), with the SM clock sampled while they ran.  Measured once per process."""
    if not _PEAKS:
        from paper_2102_08514_b300 import peaks as pk
        with ClockSampler(torch.cuda.current_device()) as clk:
            res = pk.measure(torch)
        res["clocks"] = clk.summary()
        _PEAKS.update(res)
    return _PEAKS


def brick_lb(s, esz, M, a):
    """log2 brick width of axis a of the library's coefficient layout (csrc/layout.h, cosets in
    separate arrays): the brick's 32-byte address bits dealt one per axis from axis 0."""
    bits, lb, i = (32 // esz).bit_length() - 1, 0, 0
    while bits > 0:
        if i == a:
            lb += 1
        i, bits = (i + 1) % s, bits - 1
    return lb


def distinct_sectors_per_query(spline: str, pts, esz: int = 4, dims=None):
    """Mean number of distinct 32-byte sectors (bricks) a query's coefficient gathers touch: the
    gather work of one query in the library's bricked layout, which bounds random queries (each
    distinct sector is one L1 miss and one L1 -> L2 request).  With dims: the mean number of
    distinct 128-byte lines instead (one request each when the query's sites share a load
    instruction, as in the warp-cooperative gathers).  3-D box splines (one stencil per piece);
    None otherwise.  Follows the kernels' steps: nearest coset site, |y| sorted descending (signed
    permutation), the piece from the plane bits through sigma, the piece's stencil."""
    import json as _json
    from fractions import Fraction
    with open(os.path.join(ROOT, "paper_2102_08514_b300", "csrc", "generated", "splines.json")) as f:
        meta = _json.load(f)["splines"][spline]
    if meta["s"] != 3 or meta["kind"] != 0:
        return None
    D, H, cosets = meta["D"], meta["halo"], np.asarray(meta["cosets"])
    ns = max(len(pc["sites"]) for pc in meta["pieces"])
    # every piece's stencil padded to the longest with its first site (no new sector)
    sites = np.asarray([pc["sites"] + [pc["sites"][0]] * (ns - len(pc["sites"])) for pc in meta["pieces"]])
    planes = [(np.asarray(pv, dtype=np.float64), float(Fraction(e))) for pv, e in meta["planes"]]
    sigma = np.asarray(meta["sigma"])
    M = len(cosets)
    lbs = [brick_lb(3, esz, M, a) for a in range(3)]
    x = np.asarray(pts, dtype=np.float64)
    n = len(x)
    keys = []
    for k, l in enumerate(cosets):
        u = x - l
        i = np.floor(u / D + 0.5).astype(np.int64)
        y = u - D * i
        sg = np.where(y < 0, -1, 1)
        order = np.argsort(-np.abs(y), axis=1, kind="stable")
        t = -np.sort(-np.abs(y), axis=1)
        q = np.zeros(n, dtype=np.int64)
        for b, (pv, e) in enumerate(planes):
            q |= ((t @ pv - e) >= 0).astype(np.int64) << b
        site = sites[sigma[q]]                                 # n x ns x 3
        P = np.repeat((i + 2 * H)[:, None, :], ns, axis=1)
        rows = np.arange(n)
        for A in range(3):
            ax = order[:, A]
            P[rows, :, ax] += (sg[rows, ax][:, None] * site[:, :, A])
        if dims is None:
            b = np.zeros(P.shape[:2], dtype=np.int64)
            for a in range(3):
                b = b * 4096 + (P[..., a] >> lbs[a])
            keys.append(b + (k << 40))
        else:
            # bricks in row-major order of the padded coset array (csrc/layout.h), the last
            # axis fastest; cosets one after another; a line is 128 / 32 = 4 bricks
            nb = [(((dims[a] + 4 * H + (1 << lbs[a]) - 1) >> lbs[a])) for a in range(3)]
            blin = ((P[..., 0] >> lbs[0]) * nb[1] + (P[..., 1] >> lbs[1])) * nb[2] + (P[..., 2] >> lbs[2])
            keys.append((k * nb[0] * nb[1] * nb[2] + blin) >> 2)
    K = np.sort(np.concatenate(keys, axis=1), axis=1)
    return float((1 + (np.diff(K, axis=1) != 0).sum(axis=1)).mean())


def workload_description(wl, form="value_grad", storage="f32"):
    sp = SPLINES[wl.spline]
    lat = LATTICES[sp.lattice]
    what = {"value": "value", "value_grad": "value + gradient", "adjoint": "adjoint (dL/dc)"}[form]
    src = {"signal": "sampled from the Marschner-Lobb signal", "uniform": "uniform in [-1,1]",
           "normal": "standard normal"}[wl.coeffs]
    shape = " x ".join(str(d) for d in wl.dims)
    kind = f"Voronoi spline V_{sp.order}" if sp.order else f"box spline ({np.asarray(sp.xi).shape[1]} directions)"
    return (f"{wl.name}: {wl.spline} {kind} on {lat.name.upper()}, "
            f"{len(lat.cosets)} x {shape} {storage.upper()} coefficients {src}, {wl.queries} uniform random "
            f"queries in the lattice interior, {what}")


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


def recorded_capture(kernel: str):
    """(DRAM bytes per launch, L1 -> L2 request-cycle fraction, L1 data-pipe wavefront fraction,
    warp instructions per launch) from the last ncu capture of the kernel (profiles/traffic.txt),
    or Nones when the library sources changed since that capture
    (l1tex__m_l1tex2xbar_req_cycles_active and l1tex__data_pipe_lsu_wavefronts as fractions of
    their peaks, smsp__inst_executed.sum)."""
    from paper_2102_08514_b300 import build as b
    digest = b.kernel_digest()[:16]
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.txt")) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 3 and parts[0] == kernel and parts[1] == digest:
                    return (int(parts[2]), float(parts[3]) if len(parts) > 3 else None,
                            float(parts[4]) if len(parts) > 4 else None, int(parts[5]) if len(parts) > 5 else None)
    except OSError:
        pass
    return None, None, None, None


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


def run_batch(args):
    """Batched workload: 64 volumes of uneven size and mixed lattice / spline (2^20 queries each)
    plus the D4* volume (2^24 queries), one graph-replayed persistent launch per step."""
    import torch
    from paper_2102_08514_b300.binding import Batch, Interpolator
    from synth import batch_volumes

    items = []
    total_q = 0
    flops = 0.0
    vols = batch_volumes(64) + [("d4s_8dir", (48, 48, 48, 48))]
    for v, (name, dims) in enumerate(vols):
        sp = SPLINES[name]
        lat = LATTICES[sp.lattice]
        itp = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), dims, "f32")
        rng = make_rng(2106, v)
        itp.set_coeffs(torch.from_numpy(rng.uniform(-1, 1, itp.shape).astype(np.float32)).cuda())
        nq = (1 << 24) if name == "d4s_8dir" else (1 << 20)
        if args.queries:
            nq = min(nq, args.queries)
        lo, hi = interior_box(name, dims)
        pts = torch.from_numpy(uniform_points(rng, nq, lo, hi)).cuda()
        out = torch.empty(nq, device="cuda")
        items.append((itp, pts, out))
        total_q += nq
        flops += 2.0 * itp.info.fma_value_per_query * nq
    batch = Batch(items)
    tiles = batch.autotune()
    stream = torch.cuda.current_stream()
    with ClockSampler(torch.cuda.current_device()) as clk:
        total_ms, per = time_steps(torch, batch.run, args.steps, args.warmup, stream, lambda: None)
    ms = total_ms / args.steps
    achieved = flops / (ms * 1e-3) / 1e12
    pk = measured_peaks(torch)
    peak = pk["fp32_tflops"]
    line = {
        "metric": "evals/s (batched value, FP32)", "value": total_q / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded; uniform)",
        "config": {"workload": f"batch64: 64 volumes (edge lengths log-uniform in 32..256, splines bcc_linear / "
                               f"bcc_quintic / fcc_6dir / cc_7dir in turn) x 2^20 queries + d4s_8dir 2 x 48^4 x "
                               f"2^24 queries, one persistent launch for the 3-D volumes and one piece-binned launch for the 4-D one, replayed from a CUDA graph",
                   "queries": total_q, "tiles": tiles},
        "gpu_launches": 2 * args.steps, "clocks": clk.summary(),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "k_batch (3-D and 4-D)",
                     "peak_note": "FP32 FMA rate measured in this run (peaks_fma microbenchmark), of measured"},
    }
    print(json.dumps(line), flush=True)


RAY_EVALS = [0]


def time_rays(torch, itp, wl, steps, warmup, stream, barrier):
    """1024 x 1024 orthographic rays x 256 steps through the interior box (value, value + grad)."""
    from paper_2102_08514_b300.binding import interp_eval_rays, make_rays
    from synth import ray_points, ray_setup
    W = H = 1024
    S = 256
    setup = ray_setup(wl.spline, wl.dims, W, H, S)
    eu, ev = setup["eu"], setup["ev"]
    origin = setup["centre"] - setup["half_u"] * eu - setup["half_v"] * ev
    rays = make_rays(origin, (2.0 * setup["half_u"] / W) * eu, (2.0 * setup["half_v"] / H) * ev, setup["d"],
                     setup["lo"], setup["hi"], W, H, S)
    pix = np.stack(np.meshgrid(np.arange(W), np.arange(H), indexing="xy"), -1).reshape(-1, 2)
    _, valid = ray_points(setup, pix)
    RAY_EVALS[0] = int(valid.sum()) * S
    out1 = torch.empty(W * H, device="cuda")
    out4 = torch.empty(W * H * 4, device="cuda")
    res = {}
    _, per = time_steps(torch, lambda: interp_eval_rays(itp.handle, rays, out1), steps, warmup, stream, barrier)
    res["rays_value"] = statistics.mean(per)
    _, per = time_steps(torch, lambda: interp_eval_rays(itp.handle, rays, out4, with_grad=True), steps, warmup,
                        stream, barrier)
    res["rays_value_grad"] = statistics.mean(per)
    return res


def time_fit_step(torch, itp, wl, pts, pts_h, steps, warmup, stream, barrier):
    """One Adam step of the coefficient fit: set coefficients, evaluate, FP64 loss, adjoint, update."""
    from paper_2102_08514_b300.fit import mse_loss
    from paper_2102_08514_b300.binding import lattice_interp
    from synth import marschner_lobb
    lat = LATTICES[SPLINES[wl.spline].lattice]
    phys = -1.0 + pts_h.astype(np.float64) / (lat.D * np.asarray(wl.dims) / 2.0)
    y = torch.from_numpy(marschner_lobb(phys).astype(np.float32)).cuda()
    c = torch.zeros(itp.shape, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([c], lr=0.05)
    perm, pts = itp.sort_points(pts)                     # once, as the fit driver does
    y = y[perm.long()]

    def step():
        opt.zero_grad(set_to_none=False)
        mse_loss(lattice_interp(pts, c, itp), y).backward()
        opt.step()

    _, per = time_steps(torch, step, steps, warmup, stream, barrier)
    # the fit wrote its own coefficients into the handle: restore the workload's
    itp.set_coeffs(torch.from_numpy(coefficients(wl)).cuda())
    return statistics.mean(per)


class Ranks:
    """The multi-process harness: one process per GPU (torchrun), independent query shards (weak
    scaling, no data-path collective), a barrier around the timed region and the step time taken
    as the max over ranks.  backend "nccl" on GPUs; "gloo" runs the same logic on CPU (tests)."""

    def __init__(self, backend: str = "nccl"):
        import torch
        import torch.distributed as dist
        self.dist = dist
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.device = "cpu"
        if self.world > 1:
            if backend == "nccl":
                torch.cuda.set_device(self.local)
                self.device = f"cuda:{self.local}"
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            else:
                dist.init_process_group(backend)

    def query_seed(self, base: int) -> int:
        """Each rank draws its own queries."""
        return base + 1000 * self.rank

    def barrier(self):
        if self.world > 1:
            self.dist.barrier()

    def max_over_ranks(self, x: float) -> float:
        if self.world == 1:
            return x
        import torch
        t = torch.tensor([x], device=self.device, dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_throughput(self, per_rank_units: int, max_ms: float) -> float:
        """Units processed by all ranks / the slowest rank's time."""
        return self.world * per_rank_units / (max_ms * 1e-3)

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


def workload_of(args):
    """The workload named on the command line, with its spline replaced if --spline is given."""
    wl = WORKLOADS[args.workload]
    if args.spline and args.spline != wl.spline:
        if len(LATTICES[SPLINES[args.spline].lattice].L) != len(wl.dims):
            raise SystemExit(f"--spline {args.spline}: dimension differs from workload {wl.name}")
        wl = dataclasses.replace(wl, spline=args.spline)
    return wl


def run_ours(args):
    import torch

    rk = Ranks("nccl")
    rank, world = rk.rank, rk.world
    barrier, max_over_ranks = rk.barrier, rk.max_over_ranks

    from paper_2102_08514_b300.binding import Interpolator

    wl = workload_of(args)
    form = args.form or DEFAULT_FORM[wl.name]
    sp = SPLINES[wl.spline]
    lat = LATTICES[sp.lattice]
    if sp.order:
        itp = Interpolator.named(sp.name, wl.dims, args.storage)
    else:
        itp = Interpolator(np.asarray(lat.L), np.asarray(sp.xi), wl.dims, args.storage)
    s = itp.s
    c = coefficients(wl)
    tdt = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}[args.storage]
    itp.set_coeffs(torch.from_numpy(c).to(tdt).cuda())
    lo, hi = interior_box(wl.spline, wl.dims)
    n = args.queries or wl.queries
    pts_h = uniform_points(make_rng(rk.query_seed(wl.seed), 0), n, lo, hi)
    pts = torch.from_numpy(pts_h).cuda()
    out = torch.empty(n, device="cuda")
    grad = torch.empty(n, s, device="cuda")
    gout = torch.from_numpy(make_rng(wl.seed, 5).uniform(-1, 1, n).astype(np.float32)).cuda()
    dcoef = torch.zeros(itp.shape, device="cuda")
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    run_form = {"value": lambda: itp.eval(pts, out),
                "value_grad": lambda: itp.eval_grad(pts, out, grad),
                "adjoint": lambda: itp.backward(pts, gout, dcoef)}
    step = run_form[form]

    with ClockSampler(torch.cuda.current_device()) as clk:
        total_ms, per = time_steps(torch, step, args.steps, args.warmup, stream, barrier)
    clocks = clk.summary()
    total_ms = max_over_ranks(total_ms)
    ms_step = total_ms / args.steps
    value = rk.job_throughput(n, ms_step)

    # every form, same timing rules (the timed step above is one of them)
    fw = max(args.warmup, 3)
    fsteps = max(3, min(args.steps, 20))
    form_ms = {}
    for name_f, fn in run_form.items():
        _, per_f = time_steps(torch, fn, fsteps, fw, stream, barrier)
        form_ms[name_f] = statistics.mean(per_f)

    # the same queries sorted in space (interp_sort_points): sort time, value, adjoint
    from paper_2102_08514_b300.binding import interp_sort_points
    perm = torch.empty(n, device="cuda", dtype=torch.int32)
    pts_s = torch.empty_like(pts)
    _, per_s = time_steps(torch, lambda: interp_sort_points(itp.handle, pts, perm, pts_s), fsteps, fw, stream, barrier)
    form_ms["sort"] = statistics.mean(per_s)
    gout_s = gout[perm.long()]
    _, per_f = time_steps(torch, lambda: itp.eval(pts_s, out), fsteps, fw, stream, barrier)
    form_ms["value_sorted"] = statistics.mean(per_f)
    _, per_f = time_steps(torch, lambda: itp.backward(pts_s, gout_s, dcoef), fsteps, fw, stream, barrier)
    form_ms["adjoint_sorted"] = statistics.mean(per_f)

    # workload-specific forms: ray-coherent queries (bcc_quintic_128), one fitting step (fcc_6dir_128)
    if wl.name == "bcc_quintic_128" and args.storage == "f32":
        form_ms.update(time_rays(torch, itp, wl, fsteps, fw, stream, barrier))
    if wl.name == "fcc_6dir_128" and args.storage == "f32":
        form_ms["fit_step"] = time_fit_step(torch, itp, wl, pts, pts_h, fsteps, fw, stream, barrier)
    prefilter_gbs = None
    if sp.lattice == "d4":
        # Sec. 5.2's prefilter over the whole coefficient set (samples -> padded storage); its
        # algorithmic traffic is one 4-byte read and one write per site (the 25 taps hit cache)
        from paper_2102_08514_b300.binding import d4_quasi_interpolation_filter
        taps, wts = d4_quasi_interpolation_filter()
        samples = torch.from_numpy(c).cuda()
        _, per_p = time_steps(torch, lambda: itp.prefilter(samples, taps, wts), fsteps, fw, stream, barrier)
        form_ms["prefilter"] = statistics.mean(per_p)
        itp.set_coeffs(samples)
        prefilter_gbs = itp.info.coeff_count * 8 / (form_ms["prefilter"] * 1e-3) / 1e9

    # e2e: points from pinned host memory, the step, results back to pinned host memory
    pts_pin = torch.from_numpy(pts_h).pin_memory()
    pts_d = torch.empty_like(pts)
    if form == "adjoint":
        g_pin = gout.cpu().pin_memory()
        g_d = torch.empty_like(gout)
        dc_pin = torch.empty(itp.shape, pin_memory=True)
        h2d, d2h = n * s * 4 + n * 4, dcoef.numel() * 4

        def e2e_step():
            pts_d.copy_(pts_pin, non_blocking=True)
            g_d.copy_(g_pin, non_blocking=True)
            dcoef.zero_()
            itp.backward(pts_d, g_d, dcoef)
            dc_pin.copy_(dcoef, non_blocking=True)
    else:
        # the library's host-buffer entry point: chunked copies overlapping the evaluation
        from paper_2102_08514_b300.binding import interp_eval_host
        out_pin = torch.empty(n, pin_memory=True)
        grad_pin = torch.empty(n, s, pin_memory=True)
        h2d, d2h = n * s * 4, n * 4 * (1 + (s if form == "value_grad" else 0))

        def e2e_step():
            interp_eval_host(itp.handle, pts_pin, out_pin, grad_pin if form == "value_grad" else None)

    e2e_steps = max(3, min(args.steps, 10))
    e2e_ms, _ = time_steps(torch, e2e_step, e2e_steps, fw, stream, barrier)
    e2e_ms = max_over_ranks(e2e_ms) / e2e_steps
    # the copy engines' bound on the same bytes: plain pinned copies of the step's sizes, each
    # direction alone; the pipelined step overlaps the two directions and the evaluation
    hb = torch.empty(h2d // 4, pin_memory=True)
    hd = torch.empty(h2d // 4, device="cuda")
    db = torch.empty(d2h // 4, pin_memory=True)
    dd = torch.empty(d2h // 4, device="cuda")
    h2d_ms, _ = time_steps(torch, lambda: hd.copy_(hb, non_blocking=True), 3, 2, stream, barrier)
    d2h_ms, _ = time_steps(torch, lambda: db.copy_(dd, non_blocking=True), 3, 2, stream, barrier)
    side = torch.cuda.Stream()

    def both():
        # the two directions at once, on two streams (as the pipelined step runs them)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            db.copy_(dd, non_blocking=True)
        hd.copy_(hb, non_blocking=True)
        stream.wait_stream(side)
    both_ms, _ = time_steps(torch, both, 3, 2, stream, barrier)
    h2d_ms /= 3
    d2h_ms /= 3
    both_ms /= 3
    del hb, hd, db, dd
    copy_bound_ms = max(h2d_ms, d2h_ms)

    info = itp.info
    fma = info.fma_grad_per_query if form == "value_grad" else info.fma_value_per_query
    flops_per_launch = 2.0 * fma * n
    kern_ms = statistics.mean(per)
    achieved = flops_per_launch / (kern_ms * 1e-3) / 1e12
    pk = measured_peaks(torch)
    peak = pk["fp32_tflops"]
    kname = (f"{'k_eval_coop' if info.coop else 'k_eval'}<{wl.spline},{args.storage},{form}>" if form != "adjoint"
             else f"k_adjoint<{wl.spline}>")
    traffic, l1l2_frac, l1_pipe_frac, warp_instr = recorded_capture(kname)
    esz = 4 if args.storage == "f32" else 2
    sectors = distinct_sectors_per_query(wl.spline, pts_h[:1 << 16], esz) if form != "adjoint" else None
    # L1 -> L2 requests per query: one per distinct sector when every lane gathers its own
    # query, one per distinct 128-byte line when a load instruction holds one query's sites
    lines = (distinct_sectors_per_query(wl.spline, pts_h[:1 << 16], esz, dims=wl.dims)
             if form != "adjoint" and info.coop else None)
    requests = lines if lines else sectors
    presort = presort_applies(info, n)
    if presort:
        kname += " after the piece pre-sort (whole call timed)"
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
        "data": "synthetic (seeded; " + ("Marschner-Lobb samples" if wl.coeffs == "signal" else wl.coeffs)
                + ", uniform random queries)",
        "config": {"workload": workload_description(wl, form, args.storage), "queries_per_gpu": n,
                   "coeffs": list(itp.shape), "storage": args.storage,
                   "parallelism": f"replicas x{world} (independent queries)",
                   "l2": f"inputs larger than L2 (points {n * s * 4 / 1e6:.0f} MB per GPU)" if n * s * 4 > 126e6
                   else f"inputs {n * s * 4 / 1e6:.0f} MB (smaller than L2)"},
        "e2e": {"value": world * n / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "copy_bound": {"h2d_gb_per_s": h2d / (h2d_ms * 1e-3) / 1e9, "d2h_gb_per_s": d2h / (d2h_ms * 1e-3) / 1e9,
                               "ms": copy_bound_ms, "frac": copy_bound_ms / e2e_ms,
                               "both_directions_at_once_ms": both_ms, "frac_of_both": both_ms / e2e_ms,
                               "note": "plain pinned copies of the step's bytes: the larger of the two directions "
                                       "alone, and both directions at once on two streams"}},
        "gpu_launches": args.steps * launches_per_step(form, n, presort, adjoint_bins_apply(info, n)),
        "clocks": clocks,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": kname,
                     "flops_per_query": 2.0 * fma,
                     "flops_note": "FP32 operations of the method per query (generator count: nonzeros of A_j plus "
                                   "the Horner steps on structurally nonzero data, summed over the cosets), 2 FLOP each",
                     "peak_note": f"FP32 FMA rate measured in this run (peaks_fma microbenchmark, "
                                  f"{pk['sms']} SMs, SM clock {pk['clocks']['sm_mhz']} MHz), of measured",
                     # random queries: the coefficient gathers in L1TEX beside the FP32 pipe: the
                     # L1 -> L2 requests a query makes against the measured rate of random
                     # one-sector requests (0.99 per SM clock)
                     "binding_resource": {
                         "name": ("coefficient gathers: L1 -> L2 requests per query (distinct 128-byte lines: "
                                  "one query's sites per load instruction)" if lines else
                                  "coefficient gathers: L1 -> L2 requests per query (distinct 32-byte sectors)"),
                         "sectors_per_query": sectors,
                         "lines_per_query": lines,
                         "requests_per_query": requests,
                         "achieved_grequests_s": requests * n / (kern_ms * 1e-3) / 1e9 if requests else None,
                         "peak_grequests_s": pk["gather_gsectors_s"],
                         "frac": requests * n / (kern_ms * 1e-3) / 1e9 / pk["gather_gsectors_s"] if requests else None,
                         "peak_note": "random 4-byte gathers from a 16 MiB L2-resident buffer (one request each), "
                                      "measured in this run",
                         "ncu_l1_to_l2_request_cycles_frac": l1l2_frac,
                         "ncu_l1_data_pipe_wavefronts_frac": l1_pipe_frac,
                         # the issue roofline: the recorded warp instructions of one launch over
                         # this run's kernel time, against 4 warp instructions per SM and clock
                         "instructions_per_query": warp_instr * 32 / n if warp_instr else None,
                         "issue_frac": (warp_instr / (kern_ms * 1e-3)
                                        / (4 * pk["sms"] * pk["clocks"]["sm_mhz"] * 1e6)) if warp_instr else None,
                         # every coefficient is one L1 lookup (hit or miss): against the measured
                         # rate of random L1-hit gathers
                         "l1_lookups_per_query": info.lookups_per_query,
                         "l1_lookup_frac": info.lookups_per_query * n / (kern_ms * 1e-3) / (pk["gather4B_l1_gloads_s"] * 1e9)
                         if form != "adjoint" else None,
                         # the same sectors as bytes through L2 (32 B each) against the measured
                         # coalesced L2 read rate: the bandwidth roofline of the gathers
                         "l2_gbs": sectors * 32 * n / (kern_ms * 1e-3) / 1e9 if sectors else None,
                         "l2_frac": sectors * 32 * n / (kern_ms * 1e-3) / 1e9 / pk["l2_read_gbs"] if sectors else None}},
        "peaks": {k: pk[k] for k in ("sms", "fp32_tflops", "gather_gsectors_s", "gather4B_l1_gloads_s",
                                     "gather_line2_gsectors_s", "gather_line4_gsectors_s", "red_gatomics_s",
                                     "shared_atomic_f32_gops_s", "l2_read_gbs", "tc_tf32_tflops", "clocks")},
        "forms": {k: {"evals_per_s": (RAY_EVALS[0] if k.startswith("rays") else n) / (v * 1e-3), "ms": v}
                  for k, v in form_ms.items()},
    }
    if prefilter_gbs is not None:
        line["forms"]["prefilter"] = {"ms": form_ms["prefilter"], "sites": int(itp.info.coeff_count),
                                      "gb_per_s": prefilter_gbs, "hbm_frac_of_measured": prefilter_gbs / peaks()[0]["hbm_gbs"]}
    line["forms"]["value"]["tflops"] = 2.0 * info.fma_value_per_query * n / (form_ms["value"] * 1e-3) / 1e12
    line["forms"]["value_grad"]["tflops"] = 2.0 * info.fma_grad_per_query * n / (form_ms["value_grad"] * 1e-3) / 1e12
    for k in ("rays_value", "rays_value_grad"):
        # ray-coherent samples hit L1 / L2, so the FP32 pipe is their binding roofline
        if k in form_ms:
            fma_s = info.fma_value_per_query if k == "rays_value" else info.fma_grad_per_query
            line["forms"][k]["tflops"] = 2.0 * fma_s * RAY_EVALS[0] / (form_ms[k] * 1e-3) / 1e12
    if "value_sorted" in form_ms:
        line["forms"]["value_sorted"]["tflops"] = 2.0 * info.fma_value_per_query * n / (form_ms["value_sorted"] * 1e-3) / 1e12
    for k in ("value", "value_grad", "value_sorted", "rays_value", "rays_value_grad"):
        if k in line["forms"] and "tflops" in line["forms"][k]:
            line["forms"][k]["frac_of_fp32_peak"] = line["forms"][k]["tflops"] / peak
    # the adjoint's contributions (query, site) against the measured rate of random L2 atomics
    # (the bound of a scatter with one global atomic per contribution)
    contrib = info.lookups_per_query * n
    line["forms"]["adjoint"]["contributions_per_s"] = contrib / (form_ms["adjoint"] * 1e-3)
    line["forms"]["adjoint"]["over_l2_atomic_peak"] = contrib / (form_ms["adjoint"] * 1e-3) / (pk["red_gatomics_s"] * 1e9)
    line["forms"]["adjoint"]["over_value"] = form_ms["adjoint"] / form_ms["value"]
    # the binned adjoint sums the contributions with shared-memory float atomics: their measured rate
    line["forms"]["adjoint"]["over_shared_atomic_peak"] = (contrib / (form_ms["adjoint"] * 1e-3)
                                                           / (pk["shared_atomic_f32_gops_s"] * 1e9))
    if args.workload != WORKLOAD or args.storage != "f32" or form != DEFAULT_FORM[WORKLOAD] or args.spline:
        line["metric"] = f"evals/s ({form}, {args.storage} storage)"
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], (m, ref_v, ref_g) = cpu_baseline(wl, pts_h, c, form, seconds=args.cpu_seconds)
        if form != "adjoint":
            run_form[form]()
            torch.cuda.synchronize()
            got_v = out[:m].double().cpu().numpy()
            err = got_v - ref_v
            cmax = float(np.abs(c).max())
            acc = {"sample": m, "max_abs_value": float(np.abs(err).max()), "rms_value": float(np.sqrt((err ** 2).mean())),
                   "max_abs_over_max_c": float(np.abs(err).max()) / cmax, "tolerance_over_max_c": 2e-6,
                   "against": "FP64 oracle on the original coefficients"}
            if ref_g is not None and form == "value_grad":
                eg = grad[:m].double().cpu().numpy() - ref_g
                # a C^0 spline's gradient jumps across its mesh planes: a query within FP32
                # rounding of a plane may take the other side's gradient.  Such points (the oracle's
                # own gradients 2^-14 to either side differ) are counted, not compared.
                bad = np.where(np.abs(eg).max(axis=1) > 1e-4)[0]
                crease = np.array([], dtype=np.int64)
                if len(bad):
                    orc, spl, lat_o = _oracle_setup(wl)
                    P = pts_h[bad].astype(np.float64)
                    dlt = 2.0 ** -14 * 0.5 ** np.arange(s)
                    _, g1 = orc.eval_sum(spl, lat_o.D, lat_o.cosets, c.astype(np.float64), P + dlt, grad=True)
                    _, g2 = orc.eval_sum(spl, lat_o.D, lat_o.cosets, c.astype(np.float64), P - dlt, grad=True)
                    crease = bad[np.abs(g1 - g2).max(axis=1) > 1e-3]
                keep = np.setdiff1d(np.arange(m), crease)
                acc["max_abs_grad"] = float(np.abs(eg[keep]).max())
                acc["rms_grad"] = float(np.sqrt((eg[keep] ** 2).mean()))
                acc["grad_points_at_a_crease"] = int(len(crease))
            line["accuracy"] = acc
    if rank == 0:
        print(json.dumps(line), flush=True)
    rk.close()


# ----------------------------------------------------------------------------- the oracle (CPU)

class _VoronoiOracle:
    """The oracle's Voronoi-spline methods under the module functions' call form."""

    @staticmethod
    def eval_sum(spl, *a, **k):
        return spl.eval_sum(*a, **k)

    @staticmethod
    def adjoint(spl, *a, **k):
        return spl.adjoint(*a, **k)


def _oracle_setup(wl):
    import oracle
    sp = SPLINES[wl.spline]
    lat = LATTICES[sp.lattice]
    xi = np.asarray(sp.xi)
    if sp.order:
        from fractions import Fraction
        gens = [tuple(Fraction(int(v), 2) for v in col) for col in xi.T]
        return _VoronoiOracle, oracle.VoronoiSpline(lat.L, gens, sp.order), lat
    detl = abs(round(np.linalg.det(np.asarray(lat.L, dtype=float))))
    return oracle, oracle.Spline(xi, detl), lat


def cpu_baseline(wl, pts, c, form="value_grad", seconds=15.0):
    """Time the FP64 oracle (as it stands) on the host cores on a bounded sample."""
    orc, spl, lat = _oracle_setup(wl)
    cores = os.cpu_count() or 1
    cd = c.astype(np.float64)
    # grow the sample until it takes about `seconds` (bounded), then report the last one; the
    # oracle's outputs on the first queries also serve the accuracy report
    m = 4 * cores
    while True:
        sample = pts[:m].astype(np.float64)
        t = time.perf_counter()
        res = orc.eval_sum(spl, lat.D, lat.cosets, cd, sample, grad=(form != "value"), nthreads=cores)
        dt = time.perf_counter() - t
        if dt >= 0.5 * seconds or 2 * m > len(pts):
            break
        m = int(min(len(pts), m * max(2.0, min(8.0, seconds / max(dt, 1e-3)))))
    ref_v, ref_g = (res if form != "value" else (res, None))
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{m} of the {wl.queries} queries ({'value' if form == 'value' else 'value+grad'}, FP64, "
                      f"brute-force recurrence), {dt:.1f} s"}, (m, ref_v, ref_g)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload_of(args)
    form = args.form or DEFAULT_FORM[wl.name]
    orc, spl, lat = _oracle_setup(wl)
    cores = os.cpu_count() or 1
    c = coefficients(wl).astype(np.float64)
    lo, hi = interior_box(wl.spline, wl.dims)
    pts = uniform_points(make_rng(wl.seed, 0), 1 << 16, lo, hi).astype(np.float64)
    def call(sl):
        if form == "adjoint":
            orc.adjoint(spl, lat.D, lat.cosets, c.shape, sl, np.ones(len(sl)))
        else:
            orc.eval_sum(spl, lat.D, lat.cosets, c, sl, grad=(form != "value"), nthreads=cores)

    # size each step so the whole run takes about two and a half minutes.  The oracle deals
    # queries to its threads in chunks of 4, so a sample is a multiple of unit = 4 x cores (a
    # smaller one leaves threads idle); a call on m queries costs about a + b m, fitted from two
    # probes after an untimed first call, and a step takes as many units as its share allows
    unit = 4 * cores
    call(pts[:unit])
    m1, m2 = unit, 4 * unit
    t = time.perf_counter()
    call(pts[unit:unit + m1])
    t1 = time.perf_counter() - t
    t = time.perf_counter()
    call(pts[unit + m1:unit + m1 + m2])
    t2 = time.perf_counter() - t
    b = max((t2 - t1) / (m2 - m1), 1e-7)
    a = max(t1 - b * m1, 0.0)
    budget = 150.0 / (args.steps + args.warmup)
    off = unit + m1 + m2
    units = max(1, int((budget - a) / (b * unit)))
    per_step = int(min(((len(pts) - off) // 2) // unit * unit, units * unit))

    def step(i):
        call(pts[off + (i * per_step) % (len(pts) - off - per_step):][:per_step])

    for i in range(args.warmup):
        step(i)
    t = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    dt = time.perf_counter() - t
    value = per_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC if args.workload == WORKLOAD and form == DEFAULT_FORM[WORKLOAD] and not args.spline
        else f"evals/s ({form}, {args.storage} storage)", "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": workload_description(wl, form, args.storage), "sample_per_step": per_step},
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
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch64"], default=WORKLOAD)
    ap.add_argument("--form", choices=["value", "value_grad", "adjoint"], default=None)
    ap.add_argument("--storage", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--queries", type=int, default=0, help="override the workload's query count")
    ap.add_argument("--spline", choices=sorted(SPLINES), default=None,
                    help="evaluate another spline of the same dimension on the workload's grid and queries")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
