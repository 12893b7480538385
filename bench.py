#!/usr/bin/env python3
"""Throughput of randomized resolvent analysis on one GB300 (or N, sharded).

Workload: linearised isothermal Navier-Stokes (rho, u, v) about the synthetic
separated base flow (tanh shear layer + Gaussian recirculation bubble),
Re = 500, M = 0.3, sponge on the outer 10 %, grid 512 x 256 (N = 393,216,
block 768), 64 frequencies log-spaced in [0.1, 5], k = 32 base-flow-weighted
Gaussian columns (Eq. 9).  One step = Algorithm 1 for a batch of F
frequencies: block factorisation (complex FP32), sketch + FP64 refinement to
residual <= 1e-10, FP64 CholeskyQR2, adjoint solve, small SVD, recovery
solve.  Synthetic data; the factors (~4.8 GB per frequency) exceed L2, so no
flush is needed between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
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

HBM_PEAK_GBS = 6800.0       # profiling-recipe fallback (no MEASURED_PEAKS.json)
BF16_PEAK_TFLOPS = 1900.0   # fallback burst figure
# DRAM bytes (read + write) per launch of the timed kernel class from an ncu
# capture of the current kernels (profiles/), or None when the kernel changed
# since the counters were taken.
UPDATE_TRAFFIC = None
# sweep_tc2_kernel, one launch over all 64 frequencies (profiles/sweep_tc2_ns2d-8x256-k32_batch64.md)
SWEEP_TRAFFIC = 310.0e6 + 18.3e6
PRECISIONS = ("fp32", "fp32_bf16x3", "fp32_bf16x6")
# tensor-core MMAs per FP32-level product of each operand split
SPLIT_MMAS = {"fp32": ("tf32", 3), "fp32_bf16x3": ("bf16", 3), "fp32_bf16x6": ("bf16", 6)}
WIDE_SLAB, WIDE_PANEL = 128, 16


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--batch", type=int, default=64, help="frequencies per step per GPU")
    p.add_argument("--fp64-batch", type=int, default=2)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-ref-full", action="store_true",
                   help="reference arm: skip the one whole-frequency oracle run")
    p.add_argument("--nx", type=int, default=512)
    p.add_argument("--ny", type=int, default=256)
    p.add_argument("--k", type=int, default=32)
    p.add_argument("--roofline-class", default="sweep", choices=["sweep", "update"],
                   help="kernel class of the reported roofline (the other goes to "
                        "roofline_other)")
    p.add_argument("--precision", default="fp32", choices=list(PRECISIONS),
                   help="operand split of the FP32 factors' tensor-core products")
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--workload", default="mixed", choices=["mixed", "batched", "gradient"],
                   help="mixed: 512x256, k=32, 64 frequencies (default); "
                        "batched: the 128-problem uneven batch as one graph; "
                        "gradient: d(sum of leading gains)/d(base flow) at 256x128")
    p.add_argument("--pipelines", type=int, default=1,
                   help="mixed: the step's frequencies split into this many factors objects, "
                        "each driven on its own stream by its own host thread, so one "
                        "pipeline's FP64 phases overlap another's tensor-core phases (the "
                        "per-class event times, and so the rooflines, then include the "
                        "other pipelines' concurrent kernels)")
    p.add_argument("--fd-directions", type=int, default=64,
                   help="gradient: random directions checked by central differences")
    p.add_argument("--tune", type=int, default=1, help="batched: autotune the plan")
    p.add_argument("--breakdown", action="store_true",
                   help="one extra profiled step with every kernel class timed")
    return p.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return (float(d.get("hbm_gbs", HBM_PEAK_GBS)),
                    float(d.get("bf16_tflops", BF16_PEAK_TFLOPS)), "measured")
        except Exception:
            pass
    return HBM_PEAK_GBS, BF16_PEAK_TFLOPS, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg, dev=None):
    if pg is not None:
        if dev is not None:
            pg.barrier(device_ids=[dev])
        else:
            pg.barrier()


def max_over_ranks(pg, x: float, device) -> float:
    if pg is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def batch_for(step, rank, world, F, omegas, seed0):
    """Frequencies and seeds of one step on one rank (weak scaling shards)."""
    base = (step * world + rank) * F
    idx = [(base + j) % len(omegas) for j in range(F)]
    return 1j * omegas[idx], [seed0 + i for i in idx], idx


def wide_gemm_work(b):
    """Algorithmic work of the updates of one Schur-block inverse (block b) in
    the wide factorisation.  Per 128-column slab: the rank-16 updates of the
    slab's other columns (inner: FP32 CUDA cores) and the rank-128 update of
    the columns outside it (outer: tensor cores).  Returns
    {"inner": (flops, bytes), "outer": (flops, bytes)} -- 8 real flops per
    complex multiply-add; bytes = one read and one write of every updated
    complex FP32 entry of the work matrix (the operands stream from L2)."""
    inner = [0, 0]
    outer = [0, 0]
    for c0 in range(0, b, WIDE_SLAB):
        w = min(WIDE_SLAB, b - c0)
        for k0 in range(c0, c0 + w, WIDE_PANEL):
            nbk = min(WIDE_PANEL, c0 + w - k0)
            inner[0] += 8 * b * (w - nbk) * nbk
            inner[1] += 16 * b * (w - nbk)
        if b > w:
            outer[0] += 8 * b * (b - w) * w
            outer[1] += 16 * b * (b - w)
    return {"inner": tuple(inner), "outer": tuple(outer)}


def factor_flops(b):
    """Gauss-Jordan inverse of one b x b complex block: b eliminations, each
    updating b rows x (b - 1) other columns (8 real flops per complex
    multiply-add)."""
    return 8 * b * b * (b - 1)


def metric_name(g, k):
    """The headline metric, shared by both arms so their lines compare."""
    return f"resolvent frequencies/sec at N={g.n:,}, k={k}"


def workload_config(g, k, world):
    """The workload both arms run (the implementations differ, the work does not)."""
    return {"workload": f"ns2d-{g.nx}x{g.ny}-k{k}", "N": g.n, "block": g.b, "k": k,
            "omega": "64 log-spaced in [0.1, 5]", "phi_weighted": True,
            "l2": "inputs larger than L2 (factors 4.8 GB per frequency at 512x256)",
            "parallelism": f"frequency shards x{world}"}


# ---------------------------------------------------------------- CPU oracle
def cpu_oracle_sample(grid_full, k, nx_sample, omega, seed):
    """Time the FP64 oracle (banded LAPACK LU, Householder QR, LAPACK SVD) on
    the first nx_sample streamwise columns of the workload's grid (same block
    size), returning seconds; its cost is linear in nx."""
    from oracle import operator as op
    from oracle import resolvent as rs
    g = W.Grid(kind=grid_full.kind, nx=nx_sample, ny=grid_full.ny,
               x0=grid_full.x0, x1=grid_full.x0 + (grid_full.x1 - grid_full.x0)
               * (nx_sample + 1) / (grid_full.nx + 1),
               y0=grid_full.y0, y1=grid_full.y1, re=grid_full.re, mach=grid_full.mach,
               sponge_max=grid_full.sponge_max, sponge_frac=grid_full.sponge_frac)
    flow = W.shear_bubble_flow(g)
    L = op.assemble(g, flow)
    phi = op.phi(g, flow)
    t0 = time.perf_counter()
    rs.randomized(L, 1j * omega, k, seed, phi=phi, method="banded")
    return time.perf_counter() - t0


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands on the host cores.
    Each step is a bounded sample of the workload -- one frequency's banded
    Algorithm 1 on the first nx_s of the 512 streamwise columns (same block,
    same k), 1/32 of a frequency's work since the cost is linear in the
    column count -- so ms_per_step is the measured time of that sample and
    value = (nx_s / nx) frequencies per step / step time.  After the timed
    steps one whole frequency (all 512 columns) is timed once as a check of
    that linear scaling (about 1.5 min, 15 GB of host memory)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = W.config_mixed()
    g = W.ns_grid(args.nx, args.ny)
    nx_s = 16
    times = []
    for s in range(args.warmup + args.steps):
        t = cpu_oracle_sample(g, args.k, nx_s, float(wl.omegas[s % len(wl.omegas)]), 1000 + s)
        if s >= args.warmup:
            times.append(t)
    t_step = statistics.mean(times)
    frac = nx_s / g.nx
    value = frac / t_step
    full = None
    if not args.no_ref_full:
        t_full = cpu_oracle_sample(g, args.k, g.nx, float(wl.omegas[0]), 1000)
        full = {"seconds": t_full, "frequencies_per_s": 1.0 / t_full,
                "sample_scaled_s": t_step / frac,
                "note": f"one whole frequency (all {g.nx} columns), timed once after the steps"}
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": metric_name(g, args.k),
        "value": value, "unit": "frequencies/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(g, args.k, world),
        "precision": "fp64 CPU oracle (banded LAPACK LU, Householder QR, LAPACK SVD)",
        "frequencies_per_step": frac,
        "cpu_baseline": {"value": value, "unit": "frequencies/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"each step one frequency's Algorithm 1 on the first {nx_s} of "
                                   f"{g.nx} streamwise columns (block {g.b}, banded LAPACK LU), "
                                   f"{frac:.4f} of a frequency's work (cost linear in the columns)"},
        "full_frequency": full,
        "e2e": {"value": value, "unit": "frequencies/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_1902_01458_gb300 import build as rrbuild
    if rank == 0:
        rrbuild.build()
    barrier(pg, local)
    rrbuild.build()
    import paper_1902_01458_gb300 as rr
    from paper_1902_01458_gb300 import _lib
    rr.load()

    wl = W.config_mixed()
    g = W.ns_grid(args.nx, args.ny)
    flow = W.shear_bubble_flow(g)
    k, F = args.k, args.batch
    stream = torch.cuda.current_stream(dev)
    op = rr.Operator(g, flow, device=local)
    phi = op.phi()

    # The step's F frequencies run as P pipelines (interleaved subsets), each
    # a factors object on its own stream driven by its own host thread: the
    # library's calls block their thread only (refinement reads residual
    # norms), so one pipeline's FP64 QR and residual phases overlap another's
    # factorisation and sweeps.
    P = max(1, min(args.pipelines, F))
    streams = [stream] + [torch.cuda.Stream(device=dev) for _ in range(P - 1)]

    def parallel(fns):
        if len(fns) == 1:
            return [fns[0]()]
        out, err = [None] * len(fns), []

        def run(j):
            try:
                with torch.cuda.stream(streams[j]):
                    out[j] = fns[j]()
            except BaseException as e:  # noqa: BLE001 - re-raised below
                err.append(e)
        th = [threading.Thread(target=run, args=(j,)) for j in range(len(fns))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if err:
            raise err[0]
        return out

    def merge(infos):
        m = dict(infos[0])
        for i in infos[1:]:
            for key in ("refine_iters", "refine_residual", "cqr_cond", "first_residual"):
                m[key] = max(m[key], i[key])
            m["refine_stagnated"] = m["refine_stagnated"] or i["refine_stagnated"]
            m["problem_solves"] += i["problem_solves"]
        return m

    def step(fas, s):
        shifts, seeds, _ = batch_for(s, rank, world, F, wl.omegas, wl.seed0)

        def one(j):
            def go():
                fas[j].refactor(shifts[j::P])
                V, sh, i1 = fas[j].sketch(k, seeds[j::P], phi)
                U, sig, i2 = fas[j].modes(V)
                return sig, sh, i1, i2
            return go
        res = parallel([one(j) for j in range(P)])
        return ([r[0] for r in res], [r[1] for r in res], merge([r[2] for r in res]),
                merge([r[3] for r in res]))

    # measured arithmetic peaks of this GPU (on-chip microbenchmarks)
    unit_peaks = {u: _lib.rr_measure_peak(u, local) for u in ("tf32", "bf16", "fp64", "fp32")}
    shifts0, _, _ = batch_for(0, rank, world, F, wl.omegas, wl.seed0)
    fa = [rr.Factors(op, shifts0[j::P], args.precision, streams[j]) for j in range(P)]
    info_last = None
    for s in range(args.warmup):
        step(fa, s)
    torch.cuda.synchronize(dev)
    barrier(pg, local)
    torch.cuda.synchronize(dev)
    roof_classes = ["sweep", "update"]
    _lib.rr_profile_start(roof_classes)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    solves_timed = 0   # block solves of one problem (Algorithm 1's three + corrections)
    with Clocks(local) as clk:
        start.record(stream)
        t0 = time.perf_counter()
        for s in range(args.steps):
            sig, sh, i1, i2 = step(fa, args.warmup + s)
            info_last = (i1, i2)
            solves_timed += i1["problem_solves"] + i2["problem_solves"]
        end.record(stream)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
    launches = _lib.rr_launch_count()
    cls_read = {c: _lib.rr_profile_read(c) for c in roof_classes}
    _lib.rr_profile_start([])
    elapsed_ms = start.elapsed_time(end)
    barrier(pg, local)
    elapsed_s = max_over_ranks(pg, elapsed_ms / 1e3, dev)
    value = F * world * args.steps / elapsed_s
    clocks = clk.summary()

    # per-class breakdown (one extra profiled step, not part of the value)
    breakdown = None
    if args.breakdown:
        allc = list(_lib.PROFILE_CLASSES)
        _lib.rr_profile_start(allc)
        step(fa, 0)
        torch.cuda.synchronize(dev)
        breakdown = {c: dict(zip(("ms", "launches"), _lib.rr_profile_read(c))) for c in allc}
        _lib.rr_profile_start([])

    # rooflines of the two largest kernel classes, timed in the timed region
    b, nx = g.b, g.nx
    hbm, bf16, src = peaks()
    unit, nmma = SPLIT_MMAS[args.precision]
    tensor_peak = unit_peaks[unit] / nmma   # FP32-level flops of the split
    rooflines = {}
    ms_sw, n_sw = cls_read["sweep"]
    if n_sw > 0 and ms_sw > 0:
        # every block solve of one problem streams G_i of each streamwise
        # column once forward and once backward (2 nx - 1 column steps) plus
        # its right-hand side, result and the K-split partial blocks
        tot_s = ms_sw / 1e3
        work = solves_timed * (2 * nx - 1) * (b * b * 8 + 3 * b * k * 8)
        ach = work / tot_s / 1e9
        rooflines["sweep"] = {
            "kernel": "sweep_tc2_kernel + sweep_combine_kernel (one streamwise column step "
                      "of the active frequencies, tcgen05)",
            "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "traffic": SWEEP_TRAFFIC, "peak_source": src,
            "traffic_note": "ncu DRAM read + write of one launch over all F frequencies "
                            "(the refinement's launches cover only the active ones)",
            "algorithmic_full_launch": F * (b * b * 8 + 3 * b * k * 8),
            "algorithmic_per_launch": work / n_sw, "launches": n_sw,
            "avg_launch_us": tot_s / n_sw * 1e6,
            "algorithmic_note": "per block solve of one problem: (2 nx - 1) x (b^2 x 8 B of "
                                "G_i + 3 b k x 8 B of vectors)"}
    ms_up, n_up = cls_read["update"]
    if n_up > 0 and ms_up > 0:
        # the factorisation's rank-128 updates: a complex contraction on the
        # tensor pipe; achieved = algorithmic flops / the class's event time
        tot_s = ms_up / 1e3
        gfl, gby = wide_gemm_work(b)["outer"]
        flops = gfl * nx * F * args.steps
        byts = gby * nx * F * args.steps
        ach = flops / tot_s / 1e12
        rooflines["update"] = {
            "kernel": f"gjw_gemm_kernel (complex rank-128 updates of the Schur-block "
                      f"inverse, tcgen05, {args.precision} operand split)",
            "bound": "tensor", "achieved": ach, "peak": tensor_peak, "unit": "TFLOP/s",
            "frac": ach / tensor_peak, "traffic": UPDATE_TRAFFIC,
            "peak_source": f"measured {unit} MMA peak {unit_peaks[unit]:.0f} TFLOP/s "
                           f"(rr_measure_peak) / {nmma} MMAs per FP32-level product",
            "algorithmic_per_launch": flops / n_up, "launches": n_up,
            "avg_launch_us": tot_s / n_up * 1e6,
            "hbm_achieved_gbs": byts / tot_s / 1e9, "hbm_frac": byts / tot_s / 1e9 / hbm,
            "hbm_peak_source": src}
    roof = rooflines.get(args.roofline_class)
    # lower bound of one frequency: the factorisation's flops at the split's
    # tensor peak plus the G_i streamed by every sweep of the block solves
    # actually run (each = forward + backward sweep; the three solves of
    # Algorithm 1 plus the per-frequency refinement corrections)
    n_solves = (info_last[0]["problem_solves"] + info_last[1]["problem_solves"]) / F
    t_fac = factor_flops(b) * nx / (tensor_peak * 1e12)
    t_sw = n_solves * 2 * nx * b * b * 8 / (hbm * 1e9)
    per_omega = {"bound_ms": (t_fac + t_sw) * 1e3, "factor_ms": t_fac * 1e3,
                 "sweeps_ms": t_sw * 1e3, "solves": n_solves,
                 "measured_ms": elapsed_s * 1e3 / (F * args.steps) * world,
                 "share_of_bound": (t_fac + t_sw) / (elapsed_s / (F * args.steps) * world)}

    # the FP64 GPU path on the same workload: warmed (its own factors object
    # refactored for each step), allocation outside the timed region
    fp64 = None
    if not args.no_fp64 and rank == 0:
        F64 = args.fp64_batch
        for f_ in fa:
            f_.close()
        shifts, seeds, idx64 = batch_for(args.warmup, 0, 1, F64, wl.omegas, wl.seed0)
        ref32 = rr.Factors(op, shifts, args.precision, stream)
        V, sh32, ia = ref32.sketch(k, seeds, phi)
        U, sig32, ib = ref32.modes(V)
        sig32 = sig32.cpu().numpy()
        sh32 = sh32.cpu().numpy()
        ref32.close()
        del V, U
        f64 = rr.Factors(op, shifts, "fp64", stream)
        V, sh64, ja = f64.sketch(k, seeds, phi)       # warm-up step
        U, sig64, jb = f64.modes(V)
        sig64 = sig64.cpu().numpy()
        sh64 = sh64.cpu().numpy()
        del V, U
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s64 in range(args.fp64_steps):
            sh_s, sd_s, _ = batch_for(args.warmup + 1 + s64, 0, 1, F64, wl.omegas, wl.seed0)
            f64.refactor(sh_s)
            V, _, _ = f64.sketch(k, sd_s, phi)
            U, _, _ = f64.modes(V)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t64 = e0.elapsed_time(e1) / 1e3
        f64.close()
        del V, U
        v64 = F64 * args.fp64_steps / t64
        ach64 = factor_flops(b) * nx * F64 * args.fp64_steps / t64 / 1e12
        fp64 = {"value": v64, "unit": "frequencies/s", "batch": F64, "steps": args.fp64_steps,
                "mixed_over_fp64": value / v64,
                "sigma_rel_err_max": float(np.max(np.abs(sig32 - sig64) / sig64)),
                "sigma_halko_rel_err_max": float(np.max(np.abs(sh32 - sh64) / sh64)),
                "omegas": [float(wl.omegas[i]) for i in idx64],
                "refine_residual_mixed": max(ia["refine_residual"], ib["refine_residual"]),
                "refine_residual_fp64": max(ja["refine_residual"], jb["refine_residual"]),
                "roofline": {"bound": "alu", "achieved": ach64, "peak": unit_peaks["fp64"],
                             "unit": "TFLOP/s", "frac": ach64 / unit_peaks["fp64"],
                             "note": "factorisation flops of the whole frequency over the "
                                     "step time, against the measured FP64 FMA peak"},
                "note": "warmed: one untimed batch, then refactor + Algorithm 1 per step"}
    else:
        for f_ in fa:
            f_.close()

    # end to end through the public API with host buffers (the same pipelines:
    # each thread builds its factors object, runs Algorithm 1 and copies its
    # frequencies' U, V and sigma to pinned host buffers)
    e2e = None
    if not args.no_e2e:
        pin = lambda *shape, dt: torch.empty(*shape, dtype=dt, pin_memory=True)  # noqa: E731
        nf = [len(range(j, F, P)) for j in range(P)]
        Uh = [pin(nf[j], g.n, k, dt=torch.complex128) for j in range(P)]
        Vh = [pin(nf[j], g.n, k, dt=torch.complex128) for j in range(P)]
        Sh = [pin(nf[j], k, dt=torch.float64) for j in range(P)]
        torch.cuda.synchronize(dev)
        barrier(pg, local)
        t0 = time.perf_counter()
        h2d = d2h = 0
        for s in range(args.steps):
            shifts, seeds, _ = batch_for(args.warmup + s, rank, world, F, wl.omegas, wl.seed0)
            op2 = rr.Operator(g, flow, device=local)
            h2d += 3 * g.npts * 8 + F * 16 + F * 8
            ph = op2.phi()

            def one(j):
                def go():
                    f2 = rr.Factors(op2, shifts[j::P], args.precision, streams[j])
                    V, sh, _ = f2.sketch(k, seeds[j::P], ph)
                    U, sig, _ = f2.modes(V)
                    Uh[j].copy_(U, non_blocking=True)
                    Vh[j].copy_(V, non_blocking=True)
                    Sh[j].copy_(sig, non_blocking=True)
                    streams[j].synchronize()
                    f2.close()
                return go
            parallel([one(j) for j in range(P)])
            d2h += sum(Uh[j].numel() * 16 + Vh[j].numel() * 16 + Sh[j].numel() * 8
                       for j in range(P))
            op2.close()
        wall_e2e = time.perf_counter() - t0
        wall_e2e = max_over_ranks(pg, wall_e2e, dev)
        e2e = {"value": F * world * args.steps / wall_e2e, "unit": "frequencies/s",
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        nx_s = 48
        t = cpu_oracle_sample(g, k, nx_s, float(wl.omegas[0]), 1000)
        cpu = {"value": (nx_s / g.nx) / t, "unit": "frequencies/s",
               "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one frequency's Algorithm 1 on the first {nx_s} of {g.nx} streamwise "
                         f"columns (block {g.b}, banded LAPACK LU), {t:.1f} s for "
                         f"{nx_s / g.nx:.4f} of a frequency's work (cost linear in the columns)"}

    if rank == 0:
        line = {
            "metric": metric_name(g, k),
            "value": value, "unit": "frequencies/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+f64", "data": "synthetic",
            "config": workload_config(g, k, world),
            "frequencies_per_step_per_gpu": F, "pipelines": P,
            "precision": f"mixed: fp32 factors, tensor-core updates and sweeps in the "
                         f"{args.precision} operand split, per-frequency fp64 refinement to "
                         f"1e-10 or the fp64 residual floor, fp64 CholeskyQR2 + Jacobi SVD",
            "roofline": roof,
            "roofline_other": {c: r for c, r in rooflines.items() if c != args.roofline_class},
            "per_omega": per_omega, "measured_peaks": unit_peaks,
            "cpu_baseline": cpu, "e2e": e2e, "fp64_path": fp64,
            "clocks": clocks, "gpu_launches": launches,
            "refine": {"iters": max(info_last[0]["refine_iters"], info_last[1]["refine_iters"]),
                       "residual": max(info_last[0]["refine_residual"],
                                       info_last[1]["refine_residual"]),
                       "first_residual": max(info_last[0]["first_residual"],
                                             info_last[1]["first_residual"]),
                       "stagnated": bool(info_last[0]["refine_stagnated"]
                                         or info_last[1]["refine_stagnated"]),
                       "block_solves_per_frequency": n_solves,
                       "target": "relative residual <= 1e-10 per column, or the FP64 "
                                 "residual floor where that lies above (a correction "
                                 "removing < 10 % of the residual stops the frequency)"},
            "wall_s_timed": wall,
        }
        if breakdown:
            line["breakdown_ms"] = breakdown
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def run_batched(args):
    """The uneven batching workload: 128 NS problems (grids 128..384 x
    64..256, k in {8, 16, 32, 64}, omega ~ U[0.1, 8]) as one batch plan (one
    captured CUDA graph per run), FP32 factors with FP64 refinement; ranks
    take every world-th problem.  Prints one JSON line."""
    import torch
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_1902_01458_gb300 import build as rrbuild
    if rank == 0:
        rrbuild.build()
    barrier(pg, local)
    rrbuild.build()
    import paper_1902_01458_gb300 as rr
    from paper_1902_01458_gb300 import _lib
    rr.load()
    spec = W.config_batched()
    mine = [p for i, p in enumerate(spec) if i % world == rank]
    ops, problems = {}, []
    for p in mine:
        if (p.nx, p.ny) not in ops:
            g = W.ns_grid(p.nx, p.ny)
            ops[(p.nx, p.ny)] = rr.Operator(g, W.shear_bubble_flow(g), device=local)
        problems.append({"op": ops[(p.nx, p.ny)], "shift": 1j * p.omega, "k": p.k,
                         "seed": p.seed})
    t0 = time.perf_counter()
    plan = rr.Batch(problems, precision="fp32", tune=bool(args.tune))
    plan_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        plan.run(stream)
    torch.cuda.synchronize(dev)
    barrier(pg, local)
    _lib.rr_profile_start([])
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    info = None
    with Clocks(local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            _, info = plan.run(stream)
        end.record(stream)
        torch.cuda.synchronize(dev)
    launches = _lib.rr_launch_count()
    elapsed_s = max_over_ranks(pg, start.elapsed_time(end) / 1e3, dev)
    value = len(spec) * args.steps / elapsed_s
    d = plan.describe()
    if rank == 0:
        line = {
            "metric": "resolvent problems/sec, 128-problem uneven batch (mixed FP32+FP64 "
                      "refinement, one CUDA graph per batch)",
            "value": value, "unit": "problems/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "c64+f64", "data": "synthetic",
            "config": {"workload": "ns2d-batch128-uneven", "problems": len(spec),
                       "grids": "nx in {128,256,384}, ny in {64,128,192,256}, q=3",
                       "k": "{8,16,32,64}", "omega": "U[0.1, 8]", "generator_seed": 1234,
                       "l2": "inputs larger than L2 (74 GB of factors)",
                       "parallelism": f"problem shards x{world}"},
            "plan": dict(d, plan_s=plan_s, tuned=bool(args.tune)),
            "clocks": clk.summary(), "gpu_launches": launches,
            "refine": info,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if pg is not None:
        pg.destroy_process_group()


def run_gradient(args):
    """The differentiation workload: J = sum over 16 frequencies of the 3
    leading gains at 256 x 128 (k = 16, two subspace iterations, FP64
    factors recomputed per 4-frequency chunk) and its gradient with respect to
    the nodal base flow (rho, U, V) through the autograd function.  One step
    = forward + backward.  After the timed steps the gradient is checked
    against central differences (h = 1e-6) of the same objective on the
    workload's random directions (error relative to the rms directional
    derivative).  Rank 0 only (a single-GPU workload)."""
    import torch
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_1902_01458_gb300 import build as rrbuild
    if rank == 0:
        rrbuild.build()
    barrier(pg, local)
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return
    import paper_1902_01458_gb300 as rr
    from paper_1902_01458_gb300 import _lib
    from paper_1902_01458_gb300.autograd import gain_objective
    rr.load()
    wl = W.config_gradient()
    g, base = wl.grid, wl.flow
    seeds = [wl.seed0 + i for i in range(len(wl.omegas))]
    kw = dict(grid=g, omegas=wl.omegas, k=wl.k, J=wl.J, seeds=seeds, chunk=wl.chunk,
              precision="fp64", power_iters=2)

    def grad_step():
        fields = [torch.tensor(a, dtype=torch.float64, requires_grad=True)
                  for a in (base.rho, base.u, base.v)]
        val = gain_objective(*fields, **kw)
        val.backward()
        return float(val.detach()), np.stack([f.grad.numpy() for f in fields])

    for _ in range(args.warmup):
        grad_step()
    torch.cuda.synchronize(dev)
    _lib.rr_profile_start([])
    with Clocks(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            val, grad = grad_step()
        torch.cuda.synchronize(dev)
        t_step = (time.perf_counter() - t0) / args.steps
    launches = _lib.rr_launch_count()
    # central differences on the workload's directions
    an, fd = [], []
    t1 = time.perf_counter()
    for d in W.gradient_directions(wl, args.fd_directions):
        def at(t):
            with torch.no_grad():
                f = [torch.tensor(a + t * dd) for a, dd in zip((base.rho, base.u, base.v), d)]
                return float(gain_objective(*f, **dict(kw, chunk=len(wl.omegas))))
        fd.append((at(wl.h) - at(-wl.h)) / (2 * wl.h))
        an.append(float(np.sum(grad * d)))
    t_fd = time.perf_counter() - t1
    an, fd = np.array(an), np.array(fd)
    scale = float(np.sqrt(np.mean(fd ** 2)))
    err = np.abs(an - fd) / scale
    rel = np.abs(an - fd) / np.maximum(np.abs(fd), 1e-300)
    line = {
        "metric": "gain-gradient evaluations/sec (16 frequencies, 256x128, k=16, J=3)",
        "value": 1.0 / t_step, "unit": "gradients/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ns2d-256x128-k16-grad", "N": g.n, "frequencies":
                   len(wl.omegas), "k": wl.k, "J": wl.J, "chunk": wl.chunk,
                   "power_iters": 2, "parallelism": "single GPU"},
        "timing": "host wall clock around forward + backward (autograd, includes the "
                  "host-side chunk loop), CUDA synchronised",
        "objective": val, "clocks": clk.summary(), "gpu_launches": launches,
        "fd_check": {"directions": int(len(fd)), "h": wl.h,
                     "max_err_over_rms": float(err.max()),
                     "median_rel_err": float(np.median(rel)),
                     "bar": "max |grad.d - FD(d)| <= 1e-5 x rms FD over the directions",
                     "passed": bool(err.max() <= 1e-5),
                     "seconds": t_fd},
    }
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "gradient":
        run_gradient(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
