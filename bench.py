#!/usr/bin/env python3
"""Benchmark of the split-step Crank-Nicolson GP propagation on GB300.

Workload (one GPU): 256^3 grid on [-12.8, 12.8)^3 (dx = 0.1), trap
(1, sqrt 2, 2), dt = 0.0005, the FP64-class path: psi held as float-float
pairs (GP_CFF), every sweep in FP32 error-free arithmetic, results within
the FP64 tolerance of the oracle.  Untimed preparation: the imaginary-time
ground state at g = 20 from the Gaussian seed, then a quench to g = 18 in
real time.  One benchmark step = 10 real-time SSCN steps plus one
observables report (the report interval), so every kernel of the path runs
inside the timed region.  psi (268 MB) is larger than L2 (129 MB).  The
native FP64 form (complex128, FP64 pipe) is measured beside it.

Metric: grid-point-steps/s (points x SSCN steps / s), whole job over all
ranks; with --gpus N > 1 each rank runs an independent replica (the path has
no exchange step) and the time is the max over ranks.

--impl reference times the FP64 CPU oracle on this host's cores on the same
workload (Gaussian start, 10 SSCN steps and one observables report per
benchmark step) and prints the same JSON line with "impl": "reference".
"""
import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "3D SSCN grid-point-steps/s & HBM roofline frac; serve p50/p99 vs plain"
UNIT = "grid-point-steps/s"
STEPS_PER_BENCH_STEP = 10

# FP64 flops per point of each kernel slot, counting +, -, x of the method's
# formulas (a complex multiply is 6, complex add 2, real x complex 2; exp and
# sincos count 1 each).  Real time: calcnu = |psi|^2 (3) + theta (3) + sincos
# (1) + complex multiply (6) = 13; one Crank-Nicolson line update = RHS (10)
# + forward elimination (10) + back substitution (8) = 28.  Imaginary time:
# calcnu with the scale = 2 + 3 + 3 + 1 + 2 = 11; sweep = 8 + 6 + 4 = 18.
FLOPS_PER_POINT = {
    1: {"sweep_x": 13 + 28, "sweep_y": 28, "sweep_z": 28},
    0: {"sweep_x": 11 + 18, "sweep_y": 18, "sweep_z": 18},
}
# Algorithmic HBM bytes per point of one sweep: read psi once, write it once.
SWEEP_BYTES_PER_POINT = {0: 32, 1: 16}          # by precision: c128, c64

# Float-float form: FP32 pipe lane-operations (an add, multiply or fused
# multiply-add on one lane counts 1) per point of each kernel slot, from the
# arithmetic of one Crank-Nicolson line update with exact back substitution
# (the window's redundant seed steps are not counted): product by a
# float-float coefficient 4 per lane, TwoSum 6, float-float add 8, complex
# product 16 per lane.  Real time: forward (kappa d, + psi, x mult) 28, back
# (x c', -) 24, output 2 v - psi normalised 13 -> 65 per lane, 130 per
# point; calcnu = |psi|^2 17 + a 4 + delta 12 + three complex products 96 +
# add 16 + normalise 6 = 151.  Imaginary time: forward 16, back 12, output 13
# -> 82 per point; calcnu 70.
FF_OPS_PER_POINT = {
    1: {"sweep_x": 151 + 130, "sweep_y": 130, "sweep_z": 130},
    0: {"sweep_x": 70 + 82, "sweep_y": 82, "sweep_z": 82},
}
HEADLINE_PRECISION = 2          # GP_CFF

SM_COUNT, SM_MAX_GHZ = 152, 2.07
# GB300 FP64: 2 FMA per clock per SM (1.26 TFLOP/s nominal = 152 x 2 x 2 x
# 2.07 GHz); the run measures it (gp_measure_peak) and uses that.
FP64_PEAK_TFLOPS = SM_COUNT * 2 * 2 * SM_MAX_GHZ / 1e3
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__,
                                 formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30, help="timed benchmark steps")
    ap.add_argument("--warmup", type=int, default=3, help="untimed benchmark steps")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--prep-max-steps", type=int, default=20000,
                    help="cap on imaginary-time ground-state steps before the quench")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="budget of the oracle CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the complex64 precision-form measurement")
    ap.add_argument("--probe", type=int, default=0, metavar="N",
                    help="profiling aid: load the Gaussian seed, run N real-time SSCN "
                         "steps of the workload, print nothing and exit")
    ap.add_argument("--probe-case", default=None,
                    help="workload name for --probe (default: the benchmark workload)")
    ap.add_argument("--probe-shape", type=int, default=None, help="TMA tile shape for --probe")
    ap.add_argument("--probe-path", type=int, default=None, help="sweep path (GP_PATH_*) for --probe")
    ap.add_argument("--probe-precision", type=int, default=None,
                    help="precision (GP_C128 0, GP_C64 1, GP_CFF 2) for --probe")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64, FP32 and packed FP32x2 multiply-add rates of "
                         "this GPU (the alu roofline denominators), print one JSON line, exit")
    return ap.parse_args()


def workload():
    from paper_1206_1361_gb300.workloads import REAL_256
    return REAL_256


def config_dict(case):
    """The workload, identical for both arms (precision is the line's dtype)."""
    return {"workload": case.name, "grid": list(case.shape), "dx": list(case.h), "dt": case.dt,
            "trap": [round(v, 6) for v in case.trap], "g": case.g, "mode": "real",
            "sscn_steps_per_bench_step": STEPS_PER_BENCH_STEP,
            "report_every": case.extra.get("report_every", 10),
            "l2": "inputs larger than L2 (psi 268 MB > 129 MB), no flush"}


# ------------------------------------------------------------------ clocks

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
REASON_NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, device_id):
        self.device_id = device_id
        self.proc = None

    def start(self):
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + CLOCK_FIELDS, "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.device_id:
                cmd += ["-i", self.device_id]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, v in zip(REASON_NAMES, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


# -------------------------------------------------------------- helpers

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


KERNEL_SOURCES = ("sscn_kernels.cu", "sscn_tma.cu", "sscn_axial.cu", "gp_batch.cu", "sscn_slab.cu",
                  "sscn_internal.h", "sscn_slab.h", "sscn_line.cuh", "sscn_coef.cuh", "sscn_accum.cuh",
                  "sscn_pair.cuh")


def kernel_source_sha(files=KERNEL_SOURCES):
    """Hash of kernel sources under csrc/.  An ncu summary names the files its
    kernels are compiled from (`kernel_sources:`) and their hash at capture
    (`kernel_source_sha:`); its traffic figure is used only while they match."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1206_1361_gb300", "csrc")
    for fn in files:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload_name):
    """DRAM bytes per launch of `kernel` from a committed ncu summary under
    profiles/, if it was taken on the current sources of that kernel; else
    None."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    for fn in sorted(os.listdir(pdir)):
        if not fn.endswith((".md", ".txt")):
            continue
        text = open(os.path.join(pdir, fn)).read()
        m = re.search(r"traffic\[%s@%s\]:\s*([0-9.eE+]+)" % (re.escape(kernel),
                                                           re.escape(workload_name)), text)
        if not m:
            continue
        m_src = re.search(r"kernel_sources:\s*(.+)", text)
        files = tuple(m_src.group(1).split()) if m_src else KERNEL_SOURCES
        m_sha = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", text)
        if m_sha and m_sha.group(1) == kernel_source_sha(files):
            return float(m.group(1))
    return None


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value, world):
    """Max of a float over ranks (the job time is the slowest rank's)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" \
        else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(local_ms, units_per_rank, world):
    """Job time = the slowest rank's time; value = the units all ranks
    processed over that time.  Returns (ms_max, units per second)."""
    ms_max = reduce_max(local_ms, world)
    return ms_max, world * units_per_rank / (ms_max / 1e3)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# -------------------------------------------------------------- oracle leg

def oracle_sample(case, psi0, seconds, max_steps=None):
    """Time the FP64 CPU oracle stepping `case` from psi0 for about `seconds`
    (at least 2 steps).  Returns (pt-steps/s, steps, threads)."""
    import oracle
    p = oracle.Params.make(case.shape, case.h, case.dt, *case.trap, case.g, case.mode)
    psi = psi0.copy()
    steps, t0 = 0, time.perf_counter()
    while True:
        oracle.step(p, psi, 1)
        steps += 1
        if steps % 10 == 0:
            oracle.observables(p, psi)
        el = time.perf_counter() - t0
        if (steps >= 2 and el >= seconds) or (max_steps and steps >= max_steps):
            break
    return case.points * steps / el, steps, oracle.get_threads()


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import oracle
    case = workload()
    p = oracle.Params.make(case.shape, case.h, case.dt, *case.trap, case.g, case.mode)
    psi = oracle.seed(p)
    for s in range(args.warmup):
        oracle.step(p, psi, STEPS_PER_BENCH_STEP)
        oracle.observables(p, psi)
    t0 = time.perf_counter()
    for s in range(args.steps):
        oracle.step(p, psi, STEPS_PER_BENCH_STEP)
        oracle.observables(p, psi)
    el = time.perf_counter() - t0
    value = case.points * args.steps * STEPS_PER_BENCH_STEP / el
    cores = oracle.get_threads()
    sample = ("FP64 CPU oracle (C, OpenMP over lines), %d^3 real time from the Gaussian "
              "seed, %d SSCN steps and one observables report per benchmark step"
              % (case.shape[0], STEPS_PER_BENCH_STEP))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": config_dict(case),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm

def timed_steps(gp, torch, ctx, stream, steps, record=None):
    """CUDA-event time (ms) of `steps` benchmark steps on the context's
    stream, bracketed by synchronisation; record(obs) after every step."""
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        gp.gp_step(ctx, STEPS_PER_BENCH_STEP)
        o = gp.gp_observables(ctx)
        if record:
            record(o)
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1)


def autotune_entry(gp, ctx, case, precision, mode):
    """Run the autotuner (autotune.tune, fresh cache) on a context and keep
    its pick: the chosen sweep path and tile shape, and the ms per SSCN step
    of the sweeps (per-kernel events) with the library's defaults and with
    the pick."""
    import tempfile
    import types
    from paper_1206_1361_gb300 import autotune

    def sweep_ms():
        kt = gp.gp_time_kernels(ctx, 5)
        return sum(v for k, v in kt.items() if k.startswith("sweep"))

    default_ms = sweep_ms()
    shim = types.SimpleNamespace(ctx=ctx, shape=tuple(case.shape), precision=precision)
    with tempfile.TemporaryDirectory() as d:
        pick = autotune.tune(shim, case.h, case.dt, mode, steps=5,
                             path=os.path.join(d, "autotune.json"))
    pick_ms = sweep_ms()
    return {"path": pick["path"], "shape": pick["shape"], "tuner_ms_per_step": pick["ms"],
            "sweeps_ms_per_step_default": default_ms, "sweeps_ms_per_step_pick": pick_ms,
            "speedup": default_ms / pick_ms}


def sweep_rooflines(gp, kt, points, precision, peaks, hbm_peak, hbm_src):
    """Roofline of the dominant sweep of a single-grid step from per-kernel
    times: the arithmetic bound of its form (FP32 lane-operations for the
    float-float form, FP64 flops for complex128; measured peaks) with the
    HBM fraction of its algorithmic bytes beside it."""
    sweeps = {k: v for k, v in kt.items() if k.startswith("sweep") and v > 0}
    dom = max(sweeps, key=sweeps.get)
    bpp = SWEEP_BYTES_PER_POINT[0]
    hbm_achieved = bpp * points / (sweeps[dom] * 1e-3) / 1e9
    if precision == gp.GP_CFF:
        ops = FF_OPS_PER_POINT[gp.GP_REAL]
        peak = peaks["fp32x2_fma"]["tflops"] / 2
        peak_src = ("measured FP32 pipe rate (gp_measure_peak, packed FFMA2, %.1f TFLOP/s = "
                    "%.1f T lane-operations/s)" % (peaks["fp32x2_fma"]["tflops"], peak))
        convention = "FP32 lane-operations (add, multiply or fused multiply-add on one lane = 1)"
    else:
        ops = FLOPS_PER_POINT[gp.GP_REAL]
        peak = peaks["fp64_fma"]["tflops"]
        peak_src = "measured FP64 pipe rate (gp_measure_peak, DFMA)"
        convention = "FP64 flops of the method's formulas"
    achieved = ops[dom] * points / (sweeps[dom] * 1e-3) / 1e12
    return {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": peak_src,
            "op_convention": convention, "ops_per_point": ops[dom],
            "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_achieved / hbm_peak, "peak_source": hbm_src,
                    "bytes_per_point": bpp},
            "step_hbm_frac": (3 * bpp * points / 1e9) / (sum(sweeps.values()) * 1e-3) / hbm_peak,
            "kernel_ms": {k: round(v, 5) for k, v in kt.items()}}


def run_ours(args):
    import numpy as np
    import torch

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1206_1361_gb300 import gp
    from paper_1206_1361_gb300.workloads import convergence_interval

    case = workload()
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    peaks = alu_peaks(gp)
    mp = measured_peaks()
    hbm_peak = mp.get("hbm_gbs")
    hbm_src = "measured" if hbm_peak else "fallback"
    hbm_peak = hbm_peak or FALLBACK_HBM_GBS
    g0 = case.extra["g_ground"]
    prec = HEADLINE_PRECISION
    ctx = gp.gp_create(case.shape, case.h, case.dt, *case.trap, g0, gp.GP_IMAG, prec, stream)
    try:
        # ground state at g = 20 (untimed), |dmu| < 1e-6 between checks or the cap
        gp.gp_load(ctx, None)
        k = convergence_interval(case.dt)
        mu_prev, dmu, prep = None, None, 0
        while prep < args.prep_max_steps:
            gp.gp_step(ctx, k)
            prep += k
            mu = gp.gp_observables(ctx)["mu"]
            if mu_prev is not None:
                dmu = abs(mu - mu_prev)
                if dmu < 1e-6:
                    break
            mu_prev = mu
        gp.gp_set_params(ctx, case.g, gp.GP_REAL)
        obs0 = gp.gp_observables(ctx)
        ground = torch.empty(case.points, dtype=torch.complex128, device="cuda")
        gp.gp_store(ctx, ground)

        def bench_step():
            gp.gp_step(ctx, STEPS_PER_BENCH_STEP)
            return gp.gp_observables(ctx)

        # the autotuner picks the tile shape for this grid (state restored)
        tuned = autotune_entry(gp, ctx, case, prec, gp.GP_REAL)
        for _ in range(args.warmup):
            bench_step()

        dev_id = None
        try:
            dev_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
        except Exception:
            pass
        clocks = ClockSampler(dev_id)
        rms_t = []
        barrier(world)
        clocks.start()
        ms = timed_steps(gp, torch, ctx, stream, args.steps, lambda o: rms_t.append(o["rms_r"]))
        clk = clocks.stop()
        barrier(world)
        ms_max, value = aggregate(ms, args.steps * STEPS_PER_BENCH_STEP * case.points, world)
        obs_end = gp.gp_observables(ctx)
        per_step, per_obs = gp.gp_launches_per_step(ctx)
        launches = args.steps * (STEPS_PER_BENCH_STEP * per_step + per_obs)

        # per-kernel durations (events between launches on the context stream)
        kt = gp.gp_time_kernels(ctx, 20)
        roofline = sweep_rooflines(gp, kt, case.points, prec, peaks, hbm_peak, hbm_src)
        roofline["traffic"] = profiled_traffic(roofline["kernel"], case.name + "-ff")
        roofline["autotune"] = tuned

        # end to end through the C ABI with host buffers: every step's input
        # psi (complex128) comes from pinned host memory and its observables
        # come back to the host.  The next step's input crosses to the device
        # on a second stream while the current step computes (two staging
        # buffers; the context's stream waits for the copy before gp_load
        # takes it), as a serving loop would overlap them.
        host = torch.empty(case.points, dtype=torch.complex128, pin_memory=True)
        gp.gp_store(ctx, host)
        e2e_steps = max(3, min(args.steps, 10))
        copy_stream = torch.cuda.Stream()
        stage = [torch.empty(case.points, dtype=torch.complex128, device="cuda") for _ in range(2)]
        ready = [torch.cuda.Event() for _ in range(2)]

        def h2d(b):
            with torch.cuda.stream(copy_stream):
                stage[b].copy_(host, non_blocking=True)
                ready[b].record(copy_stream)

        bench_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d(0)
        for k in range(e2e_steps):
            b = k % 2
            if k + 1 < e2e_steps:
                # stage[1 - b] last fed step k - 1, whose observables (a
                # synchronising read) have returned
                h2d(1 - b)
            stream.wait_event(ready[b])
            gp.gp_load(ctx, stage[b])
            bench_step()
        e2e_s = time.perf_counter() - t0
        e2e_s = reduce_max(e2e_s, world)
        e2e_value = world * e2e_steps * STEPS_PER_BENCH_STEP * case.points / e2e_s
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": case.points * 16,
               "d2h_bytes_per_step": 9 * 8}

        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            psi0 = host.numpy().reshape(case.shape[::-1]).copy()
            v, n, cores = oracle_sample(case, psi0, args.cpu_seconds)
            import oracle
            oracle.set_threads(1)
            v1, n1, _ = oracle_sample(case, psi0, min(4.0, args.cpu_seconds))
            oracle.set_threads(cores)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "FP64 CPU oracle, %d SSCN steps of the same 256^3 real-time "
                             "state, observables every 10th" % n,
                   "single_core": {"value": v1, "steps": n1}}

        forms = None
        if world == 1 and not args.no_forms:
            forms = {"fp64_native": fp64_native_form(gp, torch, stream, case, ground, args,
                                                     peaks, hbm_peak, hbm_src, value)}
            forms.update({"precision": precision_form(gp, torch, stream, args),
                          "batched": batched_form(gp), "serving": serving_form(gp),
                          "splitting": splitting_form(gp, torch, stream),
                          "axial": axial_form(gp, torch, stream),
                          "slab": slab_form(gp, torch, stream)})

        run = {"prep_imag_steps": prep, "prep_dmu": dmu,
               "norm_drift": abs(obs_end["norm"] / obs0["norm"] - 1),
               "rms_r_range": [min(rms_t), max(rms_t)] if rms_t else None,
               "parallelism": "replicas" if world > 1 else "single",
               "form": "float-float psi (FP32 pairs, about 48 significant bits), FP32 "
                       "error-free arithmetic, FP64 tables and reductions; parity with the "
                       "FP64 oracle <= 1e-10 over the 2000-step quench (tests)",
               "kernel_source_sha": kernel_source_sha(), "alu_peaks": peaks}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32x2 (float-float)", "data": "synthetic", "config": config_dict(case),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
                "gpu_launches": launches, "run": run, "forms": forms}
        if rank == 0:
            print(json.dumps(line), flush=True)
    finally:
        gp.gp_destroy(ctx)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    return 0


def fp64_native_form(gp, torch, stream, case, ground, args, peaks, hbm_peak, hbm_src, ff_value):
    """The same workload on the native FP64 form (complex128 psi, FP64 pipe):
    the quench from the same ground state, the benchmark's step, its
    throughput and the FP64-pipe roofline of its dominant sweep."""
    ctx = gp.gp_create(case.shape, case.h, case.dt, *case.trap, case.g, gp.GP_REAL, gp.GP_C128,
                       stream)
    try:
        gp.gp_load(ctx, ground)
        for _ in range(2):
            gp.gp_step(ctx, STEPS_PER_BENCH_STEP)
            gp.gp_observables(ctx)
        steps = max(5, min(args.steps, 20))
        ms = timed_steps(gp, torch, ctx, stream, steps)
        value = steps * STEPS_PER_BENCH_STEP * case.points / (ms * 1e-3)
        kt = gp.gp_time_kernels(ctx, 10)
        roof = sweep_rooflines(gp, kt, case.points, gp.GP_C128, peaks, hbm_peak, hbm_src)
        roof["traffic"] = profiled_traffic(roof["kernel"], case.name)
        return {"workload": case.name, "value": value, "unit": UNIT,
                "ms_per_step": ms / steps, "steps": steps, "roofline": roof,
                "float_float_speedup": ff_value / value}
    finally:
        gp.gp_destroy(ctx)


def precision_form(gp, torch, stream, args):
    """The complex64 form on 512 x 512 x 256 (real time from the Gaussian
    seed, g = 50): throughput, the HBM roofline of its dominant sweep, and the
    error of every observable after 1000 steps against an FP64 GPU run of the
    same case (FP64 reductions and tables on both)."""
    from paper_1206_1361_gb300.workloads import PRECISION_512 as case
    steps = case.steps
    out = {}
    obs, psi = {}, {}
    for prec in (gp.GP_C64, gp.GP_C128):
        ctx = gp.gp_create(case.shape, case.h, case.dt, *case.trap, case.g, gp.GP_REAL, prec,
                           stream)
        try:
            gp.gp_load(ctx, None)
            gp.gp_step(ctx, 10)
            gp.gp_observables(ctx)
            tuned = autotune_entry(gp, ctx, case, prec, gp.GP_REAL) if prec == gp.GP_C64 else None
            gp.gp_load(ctx, None)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            for _ in range(steps // STEPS_PER_BENCH_STEP):
                gp.gp_step(ctx, STEPS_PER_BENCH_STEP)
                o = gp.gp_observables(ctx)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            obs[prec] = o
            dt = torch.complex64 if prec == gp.GP_C64 else torch.complex128
            buf = torch.empty(case.points, dtype=dt, device="cuda")
            gp.gp_store(ctx, buf)
            psi[prec] = buf
            rate = steps * case.points / (ms / 1e3)
            entry = {"value": rate, "unit": UNIT, "ms_per_sscn_step": ms / steps,
                     "paths": list(gp.gp_sweep_paths(ctx))}
            if tuned:
                entry["autotune"] = tuned
            if prec == gp.GP_C64:
                kt = gp.gp_time_kernels(ctx, 10)
                sweeps = {k: v for k, v in kt.items() if k.startswith("sweep") and v > 0}
                dom = max(sweeps, key=sweeps.get)
                peaks = measured_peaks()
                peak = peaks.get("hbm_gbs") or FALLBACK_HBM_GBS
                ach = SWEEP_BYTES_PER_POINT[1] * case.points / (sweeps[dom] * 1e-3) / 1e9
                entry["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                     "frac": ach / peak, "kernel": dom,
                                     "traffic": profiled_traffic(dom, case.name),
                                     "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback",
                                     "kernel_ms": {k: round(v, 5) for k, v in kt.items()},
                                     "step_hbm_frac": (3 * SWEEP_BYTES_PER_POINT[1] * case.points / 1e9)
                                     / (sum(sweeps.values()) * 1e-3) / peak}
            out["complex64" if prec == gp.GP_C64 else "complex128"] = entry
        finally:
            gp.gp_destroy(ctx)
    a, b = psi[gp.GP_C64].to(torch.complex128), psi[gp.GP_C128]
    err = {k: abs(obs[gp.GP_C64][k] - obs[gp.GP_C128][k]) / abs(obs[gp.GP_C128][k])
           for k in ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z", "rms_r")}
    err["psi_rel_l2"] = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    del psi
    return {"workload": case.name, "steps": steps, "grid": list(case.shape),
            "complex64": out["complex64"], "complex128": out["complex128"],
            "speedup_c64_over_fp64": out["complex64"]["value"] / out["complex128"]["value"],
            "rel_error_vs_fp64": err}


def splitting_form(gp, torch, stream):
    """The symmetric (Strang) splitting and a modulated g(t): its cost on the
    benchmark workload (256^3 FP64 real time, ms per SSCN step against the
    plain splitting), and what it buys: the error at T = 0.2 of a 64^3
    real-time run with g(t) = 10 + 5 cos(20 t), plain and symmetric, at two
    dt, against the symmetric run at dt / 16 (observed orders 1 and 2)."""
    from paper_1206_1361_gb300.workloads import REAL_256 as case
    out = {}
    with gp.Solver(case.shape, case.h, case.dt, *case.trap, case.g, gp.GP_REAL, gp.GP_C128,
                   stream) as s:
        s.load(None)
        for name, split in (("lie", gp.GP_SPLIT_LIE), ("strang", gp.GP_SPLIT_STRANG)):
            s.set_splitting(split)
            s.step(STEPS_PER_BENCH_STEP)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(stream)
            s.step(10 * STEPS_PER_BENCH_STEP)
            ev1.record(stream)
            torch.cuda.synchronize()
            out[name + "_ms_per_sscn_step"] = ev0.elapsed_time(ev1) / (10 * STEPS_PER_BENCH_STEP)
    out["strang_cost_ratio"] = out["strang_ms_per_sscn_step"] / out["lie_ms_per_sscn_step"]
    shape, h, T = (64, 64, 64), (0.2, 0.2, 0.2), 0.2

    def run(dt, split):
        with gp.Solver(shape, h, dt, 1.0, 1.5, 2.0, 10.0, gp.GP_REAL, gp.GP_C128, stream) as s:
            s.set_splitting(split).set_modulation(5.0, 20.0)
            s.load(None).step(int(round(T / dt)))
            return torch.from_numpy(s.psi())

    ref = run(0.004 / 16, gp.GP_SPLIT_STRANG)
    err = {}
    for name, split in (("lie", gp.GP_SPLIT_LIE), ("strang", gp.GP_SPLIT_STRANG)):
        e = [float(torch.linalg.vector_norm(run(dt, split) - ref) / torch.linalg.vector_norm(ref))
             for dt in (0.004, 0.002)]
        err[name] = {"dt": [0.004, 0.002], "rel_l2": e, "observed_order": math.log2(e[0] / e[1])}
    out["accuracy_64cubed_modulated_T0.2"] = err
    out["workload"] = case.name + " (cost); 64^3 real time, g(t) = 10 + 5 cos(20 t) (accuracy)"
    return out


def axial_form(gp, torch, stream):
    """The axially symmetric form psi(rho, z) on 1024 x 2048 points (h =
    0.0125: rho < 12.8, |z| < 12.8), trap (1, 4), real time from the seed at
    g = 100, FP64: grid-point-steps/s, the radial sweep against the FP64
    pipe, and the oracle on the host cores on a bounded sample."""
    import oracle
    nr, nz, h, dt, g = 1024, 2048, 0.0125, 1e-4, 100.0
    steps = 10 * STEPS_PER_BENCH_STEP
    with gp.Solver.axial(nr, nz, h, h, dt, 1.0, 4.0, g, gp.GP_REAL, stream) as s:
        s.load(None).step(STEPS_PER_BENCH_STEP)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        s.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / steps
        kt = gp.gp_time_kernels(s.ctx, 10)
        paths = gp.gp_sweep_paths(s.ctx)[:2]
    points = nr * nz
    rho_ms = kt["sweep_x"]
    ach = FLOPS_PER_POINT[gp.GP_REAL]["sweep_x"] * points / (rho_ms * 1e-3) / 1e12
    p = oracle.AxialParams.make(nr, nz, h, h, dt, 1.0, 4.0, g, 1)
    psi = oracle.axial_seed(p)
    t0 = time.perf_counter()
    n_cpu = 0
    while time.perf_counter() - t0 < 5.0:
        oracle.axial_step(p, psi, 2)
        n_cpu += 2
    cpu = n_cpu * points / (time.perf_counter() - t0)
    return {"workload": "axial %dx%d h=%g, trap (1, 4), g=%g, real time, FP64" % (nr, nz, h, g),
            "value": points / (ms * 1e-3), "unit": UNIT, "ms_per_sscn_step": ms,
            "kernel_ms": {"sweep_rho": round(kt["sweep_x"], 5), "sweep_z": round(kt["sweep_y"], 5)},
            "roofline": {"bound": "alu", "kernel": "sweep_rho", "achieved": ach,
                         "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                         "note": "segmented-window sweeps (calcnu pass + radial windows); "
                                 "algorithmic flops only, the windows add overlap work"},
            "sweep_paths": list(paths),
            "cpu_baseline": {"value": cpu, "unit": UNIT, "cores": oracle.get_threads(),
                             "kind": "oracle", "sample": "%d axial SSCN steps" % n_cpu}}


def slab_form(gp, torch, stream):
    """The fused x+y slab sweep (one CTA per z-plane held in shared memory)
    against the separate sweeps, on grids whose xy-plane fits one CTA: per
    SSCN step time of each, and the fused kernel's HBM roofline (psi read and
    written once for both sweeps: 16 B per point in complex64, 32 in
    complex128)."""
    from paper_1206_1361_gb300.workloads import SLAB_C64, SLAB_FP64
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") or FALLBACK_HBM_GBS
    out = {}
    for case in (SLAB_C64, SLAB_FP64):
        entry = {"grid": list(case.shape), "steps": case.steps}
        for name, path in (("separate", gp.GP_PATH_AUTO), ("slab", gp.GP_PATH_SLAB)):
            ctx = gp.gp_create(case.shape, case.h, case.dt, *case.trap, case.g, case.mode,
                               case.precision, stream)
            try:
                gp.gp_set_option(ctx, gp.GP_OPT_SWEEP_PATH, path)
                gp.gp_load(ctx, None)
                gp.gp_step(ctx, 10)
                kt = gp.gp_time_kernels(ctx, 10)
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                torch.cuda.synchronize()
                ev0.record(stream)
                gp.gp_step(ctx, case.steps)
                ev1.record(stream)
                torch.cuda.synchronize()
                ms = ev0.elapsed_time(ev1) / case.steps
                e = {"ms_per_sscn_step": ms, "value": case.points / (ms * 1e-3), "unit": UNIT,
                     "paths": list(gp.gp_sweep_paths(ctx)),
                     "kernel_ms": {k: round(v, 5) for k, v in kt.items() if v > 0}}
                if path == gp.GP_PATH_SLAB:
                    bpp = SWEEP_BYTES_PER_POINT[case.precision]
                    ach = bpp * case.points / (kt["sweep_x"] * 1e-3) / 1e9
                    e["roofline"] = {"bound": "hbm", "kernel": "sweep_xy", "achieved": ach,
                                     "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                     "bytes_per_point": bpp,
                                     "traffic": profiled_traffic("sweep_xy", case.name),
                                     "peak_source": "measured" if peaks.get("hbm_gbs") else "fallback"}
                entry[name] = e
            finally:
                gp.gp_destroy(ctx)
        entry["speedup_slab"] = entry["separate"]["ms_per_sscn_step"] / entry["slab"]["ms_per_sscn_step"]
        out[case.name] = entry
    return out


def batch_tail(stats, frac=0.9):
    """The tail of a batch solve: the wall time after `frac` of the instances
    have finished, its share of the wall time and the throughput in it.  An
    instance's steps are taken as spread evenly over its time in the batch
    (the chunks of one launch advance every active instance alike)."""
    res = sorted(stats.results, key=lambda r: r.finished)
    if not res or stats.wall <= 0:
        return None
    k = min(len(res) - 1, max(0, int(frac * len(res)) - 1))
    t_tail = res[k].finished
    tail_s = stats.wall - t_tail
    ps = 0.0
    for r in res:
        span = r.finished - r.admitted
        if r.finished > t_tail and span > 0:
            ps += r.req.inst.points * r.total_steps * (r.finished - max(r.admitted, t_tail)) / span
    return {"after_finished_fraction": frac, "tail_s": tail_s, "share_of_wall": tail_s / stats.wall,
            "instances_in_tail": len(res) - k - 1,
            "point_steps_per_s_in_tail": ps / tail_s if tail_s > 0 else None}


def batched_form(gp):
    """256 uneven imaginary-time problems (seed 3) solved to convergence in
    one batch, against the same problems solved one at a time on complex64
    single-grid contexts."""
    from paper_1206_1361_gb300 import workloads
    from paper_1206_1361_gb300.serve import solve_batch, solve_sequential
    insts = workloads.batched_instances()
    solve_batch(insts[:2], gp.GP_C64, max_steps=20)     # warm-up: first launches load the kernels
    b = solve_batch(insts, gp.GP_C64, max_steps=40000)
    seq = solve_sequential([workloads.Request(0.0, "ground", i) for i in insts], gp.GP_C64,
                           realtime=False, max_steps=40000)
    bs, ss = b.summary(), seq.summary()
    return {"workload": "256 imaginary-time instances, edges {32..128}, 25% 2D, complex64, "
                        "to |dmu| < max(1e-6, 2^-22 mu)",
            "value": bs["point_steps_per_s"], "unit": UNIT, "wall_s": bs["wall_s"],
            "points_total": sum(i.points for i in insts),
            "max_steps": max(r.total_steps for r in b.results),
            "converged": bs["converged"], "stalled": bs["stalled"],
            "sequential_c64": {"value": ss["point_steps_per_s"], "wall_s": ss["wall_s"],
                               "converged": ss["converged"], "stalled": ss["stalled"]},
            "speedup_vs_sequential": ss["wall_s"] / bs["wall_s"],
            "tail": batch_tail(b)}


SERVE_PREFIX = 1000          # requests of the 200 req/s stream served in real time
SERVE_SEQ_SAMPLE = 100       # of those, solved one at a time by plain FP64
SERVE_SUSTAINED = (5.0, 300)  # a second seeded stream at an offered load one GB300 sustains


def serving_form(gp, prefix=SERVE_PREFIX, sample=SERVE_SEQ_SAMPLE, sustained=SERVE_SUSTAINED):
    """The seeded Poisson request stream (70 % ground state, 30 % quench;
    complex64 with FP64 reductions; 120 GB cap) through the continuous-batching
    server, three ways:
    (a) the first `prefix` requests of the 200 req/s stream with real-time
        arrivals: p50 / p99 latency and throughput over all of them (this
        offers ~20x what one GB300 solves, so latency is mostly queueing);
    (b) a seeded sample of `sample` of those requests solved one at a time by
        plain FP64 single-grid solves (the comparator): throughput per
        point-step and the ratio;
    (c) a second seeded stream at `sustained[0]` req/s (`sustained[1]`
        requests), an offered load the server keeps up with, so p50 / p99
        measure service rather than queue growth."""
    import numpy as np
    from paper_1206_1361_gb300 import workloads
    from paper_1206_1361_gb300.serve import Server, solve_sequential
    keys = ("requests", "wall_s", "requests_per_s", "point_steps_per_s", "p50_latency_s",
            "p99_latency_s", "mean_latency_s", "peak_bytes", "converged", "stalled")
    reqs = workloads.request_stream(count=prefix)
    with Server(gp.GP_C64) as srv:
        a = srv.run(reqs, realtime=True).summary()
    rng = np.random.Generator(np.random.PCG64(41))
    sub = [reqs[i] for i in sorted(rng.choice(len(reqs), sample, replace=False))]
    b = solve_sequential(sub, gp.GP_C128, realtime=False).summary()
    rate, count = sustained
    reqs_c = workloads.request_stream(seed=5, count=count, rate=rate)
    with Server(gp.GP_C64) as srv:
        c = srv.run(reqs_c, realtime=True).summary()
    offered = sum(r.inst.points for r in reqs_c)
    return {"workload": ("(a) first %d requests of the seeded stream (seed 4, 200 req/s, real-time "
                         "arrivals); (b) %d of them (PCG64 seed 41) solved one at a time in plain "
                         "FP64; (c) %d requests of a second stream (seed 5) at %g req/s"
                         % (prefix, sample, count, rate)),
            "a_overload_200rps": {k: a[k] for k in keys},
            "b_sequential_fp64_sample": {k: b[k] for k in keys if k != "peak_bytes"},
            "c_sustained": dict({k: c[k] for k in keys}, offered_rps=rate,
                                arrival_span_s=reqs_c[-1].arrival,
                                offered_points=offered),
            "throughput_ratio": a["point_steps_per_s"] / b["point_steps_per_s"],
            "throughput_ratio_target": 3.0}


PROBE_BATCH = "batch-60-requests-c64"
PROBE_AXIAL = "axial-1024x2048-fp64"
# the 128 x 128 x 32 instance of the batched set alone in a batch (10-step
# launches, one more than --probe // 10): a batch's tail in miniature
PROBE_BATCH_ONE = "batch-1-128x128x32-c64"


def run_probe(args):
    """A short run of one workload for profilers: N steps after setup.
    --probe-case picks a single-grid case by name, PROBE_BATCH (the first 60
    instances of the request stream in one batch, complex64, imaginary time)
    or PROBE_AXIAL (the axial form of the bench)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1206_1361_gb300 import gp
    from paper_1206_1361_gb300.workloads import CASES, request_stream
    from paper_1206_1361_gb300.workloads import batched_instances as workloads_batched
    if args.probe_case == PROBE_BATCH:
        with gp.Batch(gp.GP_C64, 1 << 36) as b:
            for r in request_stream(count=60):
                i = r.inst
                b.add(i.shape, i.h, i.dt, *i.trap, i.g, gp.GP_IMAG)
            b.step(args.probe)
            gp.gp_batch_sync(b.b)
        torch.cuda.synchronize()
        return 0
    if args.probe_case == PROBE_BATCH_ONE:
        inst = [i for i in workloads_batched() if i.shape == (128, 128, 32)][0]
        with gp.Batch(gp.GP_C64, 1 << 34) as b:
            b.add(inst.shape, inst.h, inst.dt, *inst.trap, inst.g, gp.GP_IMAG)
            for _ in range(1 + args.probe // 10):
                b.step(10)
                gp.gp_batch_sync(b.b)
        torch.cuda.synchronize()
        return 0
    if args.probe_case == PROBE_AXIAL:
        with gp.Solver.axial(1024, 2048, 0.0125, 0.0125, 1e-4, 1.0, 4.0, 100.0, gp.GP_REAL) as s:
            s.load(None).step(args.probe).sync()
            s.observables()
        torch.cuda.synchronize()
        return 0
    case = CASES[args.probe_case] if args.probe_case else workload()
    prec = case.precision if args.probe_precision is None else args.probe_precision
    with gp.Solver(case.shape, case.h, case.dt, *case.trap, case.g, gp.GP_REAL, prec) as s:
        if args.probe_shape is not None:
            gp.gp_set_option(s.ctx, gp.GP_OPT_TILE_SHAPE, args.probe_shape)
        if args.probe_path is not None:
            s.set_path(args.probe_path)
        s.load(None).step(args.probe).sync()
        s.observables()
    torch.cuda.synchronize()
    return 0


PEAK_ITERS = {"fp64_fma": 20000, "fp32_fma": 400000, "fp32x2_fma": 200000}


def alu_peaks(gp):
    """Measured TFLOP/s of the FP64, FP32 and packed FP32x2 multiply-add pipes
    (gp_measure_peak: best of three launches over every CTA slot)."""
    kinds = {"fp64_fma": gp.GP_PEAK_FP64_FMA, "fp32_fma": gp.GP_PEAK_FP32_FMA,
             "fp32x2_fma": gp.GP_PEAK_FP32X2_FMA}
    out = {}
    for name, kind in kinds.items():
        tf, ms = gp.gp_measure_peak(kind, PEAK_ITERS[name])
        out[name] = {"tflops": tf, "ms": ms, "iters": PEAK_ITERS[name]}
    return out


def run_peaks(args):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1206_1361_gb300 import gp
    dev_id = None
    try:
        dev_id = "GPU-" + str(torch.cuda.get_device_properties(0).uuid)
    except Exception:
        pass
    clocks = ClockSampler(dev_id)
    clocks.start()
    peaks = alu_peaks(gp)
    clk = clocks.stop()
    print(json.dumps({"peaks": peaks, "clocks": clk,
                      "device": torch.cuda.get_device_name(0)}), flush=True)
    return 0


def main():
    args = parse_args()
    if args.peaks:
        return run_peaks(args)
    if args.probe:
        return run_probe(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
