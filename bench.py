"""Benchmark: ENO-AO cell-stage updates per second on the 2D Euler workload.

Workload (seeded, synthetic): 2D Euler, gamma 1.4, 4096 x 4096 cells on
[0,1]^2, transmissive boundaries, four-quadrant Riemann data (rho, p ~
U[0.1,1.5], u, v ~ U[-1,1] per quadrant, split point ~ U[0.4,0.6]^2),
dimension-by-dimension characteristic ENO-AO5, third-order TVD Runge-Kutta,
CFL 0.5.  A step is one Runge-Kutta step (three stages, both axes) over the
whole grid.  The metric compares the FP32-bulk path (reconstruction in FP32,
state and Runge-Kutta accumulation in FP64) with the all-FP64 path; the
line's value is the FP32-bulk throughput, the FP64 throughput and the L1
difference of the two states after the timed steps ride along.

Usage:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
With --impl reference the reference arm is the FP64 C oracle on the host
cores, one step per iteration on a bounded sub-block of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CELLS = 4096
CFL = 0.5
SEED = 1
METRIC = "ENO-AO cell-stage updates/s (FP64 vs FP32-mixed) + L1 err vs FP64 oracle"
FLOPS_PER_FACE = 1150       # flops of one face of one axis, 2D Euler ENO-AO5 (the method's
                            # operation count: split, Roe eigen-system, projection of both
                            # windows, indicators, selection, back-projection)
FLOPS_PER_FACE_COUNTED = 885  # the same path counted operation by operation in the kernel
# y sweep, stage 0: read U^n (FP64) and L_x (FP32), write U1 (FP64) and the
# FP32 increment I0 the later stages combine with
BYTES_PER_CELL_Y = 32 + 16 + 32 + 16
WORKLOAD = "euler2d-4096x4096-quadrant-riemann-ao5"


def max_over_ranks(ms, device):
    """Slowest rank's time (ms); the whole job takes as long as its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, ms_max, world_size):
    """Whole-job throughput: units processed by all ranks over the slowest rank's time
    (each rank advances its own replica of the workload: weak scaling)."""
    return units_per_rank * world_size / (ms_max / 1e3)


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self, t0=None, t1=None):
        """Median SM clock and the reasons seen; with t0, t1 (time.monotonic()
        around a timed region) only the samples that arrived within it."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [ln for ts, ln in self.lines]
        window = "whole run"
        if t0 is not None:
            inside = [ln for ts, ln in self.lines if t0 <= ts <= t1 + 0.15]
            if inside:
                lines, window = inside, "timed region"
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "window": window}


def workload_state():
    from paper_2108_12742_gb300 import inputs
    return inputs.euler2d_quadrants(N_CELLS, N_CELLS, seed=SEED)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0}, "fallback"


def cpu_model():
    """Model name of the host CPU (x86 'model name', else Arm implementer/part)."""
    try:
        text = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    import re
    m = re.search(r"^model name\s*:\s*(.+)$", text, re.M)
    if m:
        return m.group(1).strip()
    imp = re.search(r"^CPU implementer\s*:\s*(\S+)", text, re.M)
    part = re.search(r"^CPU part\s*:\s*(\S+)", text, re.M)
    names = {("0x41", "0xd4f"): "Arm Neoverse V2 (NVIDIA Grace)"}
    if imp and part:
        return names.get((imp.group(1), part.group(1)),
                         f"Arm implementer {imp.group(1)} part {part.group(1)}")
    return "unknown"


def measure_peaks(local):
    """FP32, packed-FP32 and FP64 multiply-add peaks of this GPU from the
    library's microbenchmark, with the SM clock sampled while it runs."""
    import paper_2108_12742_gb300 as eno
    out = {}
    clk = ClockSampler(local)
    clk.start()
    for kind, name, trips in ((eno.PEAK_FP32, "fp32", 4000), (eno.PEAK_FP32X2, "fp32x2", 2000),
                              (eno.PEAK_FP64, "fp64", 200)):
        best = 0.0
        for _ in range(3):
            tf, _ = eno.measure_fma_peak(kind, trips)
            best = max(best, tf)
        out[name] = best
    out["clocks"] = clk.stop()
    return out


def step_roofline(value, flops_per_cs, bytes_fused, bytes_split, peaks, hbm):
    """Whole-step roofline of a workload line: the method's flops per
    cell-stage (§8(d)'s count) times the line's cell-stage rate against the
    FP32 multiply-add peak measured in this run, and the bytes per cell-stage
    of an all-axes-fused design and of this per-axis design against the
    measured copy bandwidth."""
    achieved = flops_per_cs * value / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peaks["fp32"], "unit": "TFLOP/s",
            "frac": achieved / peaks["fp32"], "traffic": None,
            "flops_per_cell_stage": flops_per_cs, "kind": "whole step (every sweep of a stage)",
            "peak_kind": "measured: FP32 multiply-add microbenchmark on this GPU, 'of measured'",
            "hbm": {"peak": hbm, "unit": "GB/s",
                    "frac_fused_bytes": bytes_fused * value / 1e9 / hbm,
                    "frac_per_axis_bytes": bytes_split * value / 1e9 / hbm,
                    "bytes_per_cell_stage": {"fused": bytes_fused, "per_axis": bytes_split}}}


def profiled_traffic(summary):
    """DRAM bytes per launch of the dominant kernel at 4096^2, from the committed
    ncu summary, if that summary was taken on the current kernel source."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles", summary)
    src = os.path.join(ROOT, "paper_2108_12742_gb300", "csrc", "sweep.cuh")
    if not os.path.exists(prof):
        return None
    text = open(prof).read()
    m = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    t = re.search(r"traffic_bytes_per_launch_4096:\s*([0-9.eE+]+)", text)
    if not m or not t:
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != m.group(1):
        return None
    return float(t.group(1))


def cpu_sample(U0, sub, nthreads=0):
    """One oracle step on a sub x sub block of the workload (the full grid's
    alpha and dt), returning (cell-stage updates/s, seconds, threads)."""
    import oracle
    blk = np.ascontiguousarray(U0[:, :, :sub, :sub])
    P = oracle.make_problem((sub, sub), (0.0, 0.0), (sub / N_CELLS, sub / N_CELLS),
                            system=oracle.EULER, order=5, bc=oracle.TRANSMISSIVE,
                            nthreads=nthreads)
    full = oracle.make_problem((N_CELLS, N_CELLS), (0.0, 0.0), (1.0, 1.0), system=oracle.EULER,
                               order=5, bc=oracle.TRANSMISSIVE)
    alpha = oracle.alpha(full, U0)   # alpha is a property of the whole mesh
    dx = 1.0 / N_CELLS
    dt = CFL / (alpha[0] / dx + alpha[1] / dx)
    t0 = time.perf_counter()
    oracle.step_alpha(P, blk, dt, alpha)
    sec = time.perf_counter() - t0
    threads = nthreads if nthreads > 0 else (os.cpu_count() or 1)
    return sub * sub * 3 / sec, sec, threads


def run_reference(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return 0
    U0 = workload_state()
    sub = 512
    for _ in range(args.warmup):
        cpu_sample(U0, sub)
    secs = []
    rate = threads = None
    for _ in range(args.steps):
        rate, sec, threads = cpu_sample(U0, sub)
        secs.append(sec)
    total = sum(secs)
    value = sub * sub * 3 * args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "cell-stage updates/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": N_CELLS * N_CELLS, "order": 5, "cfl": CFL,
                   "sample": f"one step of a {sub}x{sub} sub-block per iteration",
                   "l2": "inputs larger than L2 not applicable (host run)"},
        "cpu_baseline": {"value": value, "unit": "cell-stage updates/s", "cores": threads,
                         "kind": "oracle",
                         "sample": f"one RK3 step of a {sub}x{sub} block of the 4096^2 workload"},
        "e2e": {"value": value, "unit": "cell-stage updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_gpu(args):
    import torch

    import paper_2108_12742_gb300 as eno

    ws, rank, local = _dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    U0 = workload_state()
    nbytes = U0.nbytes
    stream = torch.cuda.current_stream()
    dev_U0 = torch.from_numpy(U0).cuda()

    def make(precision):
        s = eno.Solver((N_CELLS, N_CELLS), (0.0, 0.0), (1.0, 1.0), stream=stream,
                       system=eno.EULER, order=5, bc=eno.TRANSMISSIVE, precision=precision)
        s.init_state(dev_U0)
        if args.tiles and precision == eno.FP32_BULK:
            # the FP32-bulk tiles given on the command line (profiler captures
            # use the ones a plain run's autotuner chose)
            t = [int(v) for v in args.tiles.split(",")]
            s.set_tiles(0, t[0], t[1])
            s.set_tiles(1, t[2], t[3])
        elif not args.no_autotune:
            # tiles timed on data like the timed steps': the state after 20
            # steps (the four-quadrant start has no developed flow yet);
            # the timed run starts again from the initial state
            s.advance_steps(20, CFL)
            s.autotune()
        s.init_state(dev_U0)
        return s

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(s, k):
        s.advance_steps(args.warmup, CFL)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.advance_steps_async(k, CFL)
        e1.record(stream)
        s.sync()
        barrier()
        return max_over_ranks(e0.elapsed_time(e1), "cuda")

    cells = N_CELLS * N_CELLS
    # ---- FP32-bulk (the line's value)
    s32 = make(eno.FP32_BULK)
    clk = ClockSampler(local)
    clk.start()
    ms32 = timed(s32, args.steps)
    clocks = clk.stop()
    st32 = s32.stats()
    # dominant kernel: the last-axis sweep (combine), timed alone on its stream
    k_ms32 = [s32.time_sweep(d, 5) for d in range(2)]
    # ---- FP64
    k64 = max(1, min(args.steps, args.fp64_steps))
    s64 = make(eno.FP64)
    clk64 = ClockSampler(local)
    clk64.start()
    ms64 = timed(s64, k64)
    clocks64 = clk64.stop()
    k_ms64 = [s64.time_sweep(d, 2) for d in range(2)]
    # ---- L1 difference FP32-bulk vs FP64 after the same number of steps
    s32.init_state(dev_U0)
    s64.init_state(dev_U0)
    kcmp = k64
    s32.advance_steps(kcmp, CFL)
    s64.advance_steps(kcmp, CFL)
    a = torch.empty_like(dev_U0)
    b = torch.empty_like(dev_U0)
    s32.get_state(a)
    s64.get_state(b)
    diff = (a - b).abs()
    l1 = [float(diff[v].mean() / b[v].abs().mean()) for v in range(4)]
    linf = [float(diff[v].max() / b[v].abs().max()) for v in range(4)]
    decisions = 2 * 4 * 3 * 2 * cells  # fields x signs x stages x axes per step (faces ~ cells)
    fallback_rate = st32.fp64_fallbacks / max(1, decisions * (st32.steps))
    evolved64 = b.cpu().numpy() if rank == 0 and not args.no_cpu else None

    # ---- end to end through the public API with host buffers (FP32-bulk)
    host_in = torch.from_numpy(U0).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    ke2e = max(1, min(args.steps, 10))
    s32.init_state(host_in.numpy())
    barrier()
    t0 = time.perf_counter()
    for _ in range(ke2e):
        s32.init_state(host_in.numpy())
        s32.advance_steps(1, CFL)
        s32.get_state(host_out.numpy())
    torch.cuda.synchronize()
    e2e_sec = max_over_ranks(time.perf_counter() - t0, "cuda")
    e2e_value = job_value(cells * 3 * ke2e, e2e_sec * 1e3, ws)

    value = job_value(cells * 3 * args.steps, ms32, ws)
    value64 = job_value(cells * 3 * k64, ms64, ws)

    # Roofline of the dominant FP32-bulk kernel, the y-axis sweep (largest
    # share of a step in the launch list): it adds L_x, combines and, on the
    # last stage, checks the state and takes the next alpha.  It is timed alone
    # right after the timed region on the library's stream (CUDA events on
    # that stream), stage 0 in the mode it has inside a step.  The peak is the
    # FP32 multiply-add rate measured on this GPU by the library's
    # microbenchmark.  Algorithmic work per face: FLOPS_PER_FACE (the method's
    # count), FLOPS_PER_FACE_COUNTED (the kernel's own operations) beside it;
    # bytes per cell: read U^n (4 x 8 B) and L_x (4 x 4 B), write U1 (4 x 8 B).
    peaks, peak_kind = measured_peaks()
    fma = measure_peaks(local)
    dom = 1
    t_dom = k_ms32[dom] / 1e3
    flops = FLOPS_PER_FACE * cells
    achieved = flops / t_dom / 1e12
    achieved_counted = FLOPS_PER_FACE_COUNTED * cells / t_dom / 1e12
    traffic = profiled_traffic("sweep_y_fp32_euler2d.md")
    roofline = {"bound": "alu", "achieved": achieved, "peak": fma["fp32"], "unit": "TFLOP/s",
                "frac": achieved / fma["fp32"], "traffic": traffic,
                "kernel": "sweep_kernel<4,5,float> y axis (stage 0, adds L_x, combines)",
                "peak_kind": "measured: FP32 multiply-add microbenchmark on this GPU "
                             "(enoao_measure_fma_peak), 'of measured'",
                "peak_clock_mhz": fma["clocks"].get("sm_mhz"),
                "flops_per_face": FLOPS_PER_FACE,
                "kernel_ms": k_ms32[dom], "algorithmic_flops_per_launch": flops,
                "counted": {"flops_per_face": FLOPS_PER_FACE_COUNTED,
                            "achieved": achieved_counted, "frac": achieved_counted / fma["fp32"]},
                "measured_peaks_tflops": {k: fma[k] for k in ("fp32", "fp32x2", "fp64")},
                "hbm": {"achieved": BYTES_PER_CELL_Y * cells / t_dom / 1e9,
                        "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": BYTES_PER_CELL_Y * cells / t_dom / 1e9 / peaks["hbm_gbs"],
                        "algorithmic_bytes_per_launch": BYTES_PER_CELL_Y * cells,
                        "peak_kind": peak_kind}}
    # the FP64 path's y sweep against the measured FP64 multiply-add rate
    a64 = flops / (k_ms64[dom] / 1e3) / 1e12
    roofline64 = {"bound": "fp64 alu", "achieved": a64, "peak": fma["fp64"], "unit": "TFLOP/s",
                  "frac": a64 / fma["fp64"], "kernel_ms": k_ms64[dom],
                  "peak_kind": "measured: FP64 multiply-add microbenchmark on this GPU"}

    launches = (s32.launches_per_step() * args.steps) if rank == 0 else 0

    cpu = None
    agreement = None
    if rank == 0 and not args.no_cpu:
        rate, sec, threads = cpu_sample(U0, args.cpu_sub)
        rate1, sec1, _ = cpu_sample(U0, args.cpu_sub1, nthreads=1)
        cpu = {"value": rate, "unit": "cell-stage updates/s", "cores": threads, "kind": "oracle",
               "cpu_model": cpu_model(),
               "sample": f"one RK3 step of a {args.cpu_sub}x{args.cpu_sub} block of the "
                         f"4096^2 workload ({sec:.1f} s, {threads} threads)",
               "single_thread": {"value": rate1, "unit": "cell-stage updates/s", "cores": 1,
                                 "sample": f"one RK3 step of a {args.cpu_sub1}x{args.cpu_sub1} "
                                           f"block ({sec1:.1f} s)"}}
        agreement = choice_agreement(evolved64, args.agree_sub, kcmp)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "cell-stage updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms32 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32-bulk/f64-state", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": cells, "order": 5, "cfl": CFL,
                       "seed": SEED, "parallelism": f"replicas{ws}" if ws > 1 else "single",
                       "l2": "inputs larger than L2 (537 MB state per array)",
                       "tiles": {d: s32.get_tiles(d) for d in range(2)}},
            "fp64": {"value": value64, "ms_per_step": ms64 / k64, "steps": k64,
                     "kernel_ms": k_ms64, "clocks": clocks64, "roofline": roofline64},
            "fp32_bulk_speedup_vs_fp64": value / value64,
            "l1_rel_fp32_bulk_vs_fp64": l1, "linf_rel_fp32_bulk_vs_fp64": linf,
            "compare_steps": kcmp, "fp64_fallback_rate": fallback_rate,
            "kernel_ms_fp32_bulk": k_ms32,
            "roofline": roofline, "cpu_baseline": cpu,
            "fp64_choice_agreement_vs_oracle": agreement,
            "e2e": {"value": e2e_value, "unit": "cell-stage updates/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line))
    for s in (s32, s64):
        s.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def choice_agreement(U, sub, steps):
    """Stencil choices of the FP64 GPU path against the oracle's on a sub x sub
    block of the evolved workload state (both axes, every field, sign and
    face): the agreement rate, and how many disagreements the near-tie rule
    excuses (the oracle's deciding comparison within 1e-13 of the indicators'
    magnitude) or not."""
    import oracle
    import paper_2108_12742_gb300 as eno
    if U is None:
        return None
    n = U.shape[-1]
    y0 = x0 = (n - sub) // 2  # centre block: the quadrant split runs through it
    blk = np.ascontiguousarray(U[:, :, y0:y0 + sub, x0:x0 + sub])
    h = sub / n
    P = oracle.make_problem((sub, sub), (0.0, 0.0), (h, h), system=oracle.EULER, order=5,
                            bc=oracle.TRANSMISSIVE)
    total = agree = excused = 0
    with eno.Solver((sub, sub), (0.0, 0.0), (h, h), system=eno.EULER, order=5,
                    bc=eno.TRANSMISSIVE, precision=eno.FP64) as s:
        s.init_state(blk)
        for d in range(2):
            _, idx = s.reconstruct_fluxes(d, want_idx=True)
            _, io, gap = oracle.fluxes(P, blk, d, want_idx=True)
            differ = idx != io
            total += idx.size
            agree += int((~differ).sum())
            excused += int((differ & (gap <= 1e-13)).sum())
    return {"choices": total, "agreement": agree / total, "disagreements": total - agree,
            "excused_near_ties": excused, "unexcused": total - agree - excused,
            "sample": f"{sub}x{sub} centre block of the 4096^2 state after {steps} FP64 steps, "
                      "both axes, every field, sign and face"}


# ----------------------------------------------------------------------------
# Further workloads (not the headline line): python bench.py --workload NAME
# ----------------------------------------------------------------------------
def _line(workload, value, ms_step, steps, warmup, extra):
    d = {"metric": METRIC, "value": value, "unit": "cell-stage updates/s", "n_gpus": 1,
         "steps": steps, "warmup": warmup, "ms_per_step": ms_step, "higher_is_better": True,
         "scaling": "weak", "vs_baseline": None, "dtype": "f32-bulk/f64-state",
         "data": "synthetic", "config": {"workload": workload}}
    d.update(extra)
    print(json.dumps(d))


def _timed_steps(s, k, warmup, cfl, stream):
    import torch
    s.advance_steps(warmup, cfl)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.advance_steps_async(k, cfl)
    e1.record(stream)
    s.sync()
    return e0.elapsed_time(e1)


def run_batched(args):
    """4096 independent 1D Euler problems, N ~ log-uniform[256, 16384], 200 steps
    in one persistent launch (FP32 bulk and FP64), against one launch per problem
    (timed on a random subset of the problems, scaled by their cells)."""
    import torch
    import paper_2108_12742_gb300 as eno
    from paper_2108_12742_gb300 import inputs
    clk = ClockSampler(0)
    clk.start()
    nprob, nsteps = 4096, args.batch_steps
    sizes = inputs.batch_sizes(nprob, seed=2024)
    U = inputs.batch_states(sizes, seed=10_000)
    cells = int(sizes.sum())
    stream = torch.cuda.current_stream()
    res = {}
    for name, prec in (("fp32_bulk", eno.FP32_BULK), ("fp64", eno.FP64)):
        with eno.Batch(sizes, 0.0, 1.0, stream=stream, system=eno.EULER, order=5,
                       precision=prec) as b:
            b.init_state(U)
            b.autotune()
            b.init_state(U)
            b.advance_steps(1, CFL)          # warm-up launch
            b.init_state(U)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.advance_steps_async(nsteps, CFL)
            e1.record(stream)
            b.sync()
            ms = e0.elapsed_time(e1)
            res[name] = {"value": cells * 3 * nsteps / (ms / 1e3), "ms_total": ms,
                         "state": b.get_state()}
    # one launch per problem: the single-problem path on a seeded subset
    rng = np.random.default_rng(7)
    sub = np.sort(rng.choice(nprob, size=args.batch_subset, replace=False))
    off = np.concatenate([[0], np.cumsum(sizes)])
    ms_sub, cells_sub = 0.0, 0
    for i in sub:
        n = int(sizes[i])
        with eno.Solver((n,), (0.0,), (1.0,), stream=stream, system=eno.EULER, order=5,
                        precision=eno.FP32_BULK) as s:
            s.init_state(U[:, off[i]:off[i + 1]].reshape(3, 1, 1, n))
            ms_sub += _timed_steps(s, nsteps, 0, CFL, stream)
            cells_sub += n
    per_problem = cells_sub * 3 * nsteps / (ms_sub / 1e3)
    a, b = res["fp32_bulk"]["state"], res["fp64"]["state"]
    l1 = [float(np.abs(a[v] - b[v]).mean() / np.abs(b[v]).mean()) for v in range(3)]
    clocks = clk.stop()
    mp, _ = measured_peaks()
    roof = step_roofline(res["fp32_bulk"]["value"], 760, 64, 64, measure_peaks(0), mp["hbm_gbs"])
    _line("batched-euler1d-4096-problems-N256-16384-ao5", res["fp32_bulk"]["value"],
          res["fp32_bulk"]["ms_total"] / nsteps, nsteps, 1,
          {"clocks": clocks, "config": {"workload": "batched-euler1d-4096-problems-N256-16384-ao5", "cells": cells,
                      "problems": nprob, "steps_per_launch": nsteps, "launches": 1},
           "fp64": {"value": res["fp64"]["value"], "ms_total": res["fp64"]["ms_total"]},
           "fp32_bulk_speedup_vs_fp64": res["fp32_bulk"]["value"] / res["fp64"]["value"],
           "roofline": roof,
           "one_launch_per_problem": {"value": per_problem, "problems_timed": len(sub),
                                      "cells_timed": cells_sub,
                                      "note": "single-problem path, FP32 bulk, same steps"},
           "batched_speedup_vs_per_problem": res["fp32_bulk"]["value"] / per_problem,
           "l1_rel_fp32_bulk_vs_fp64": l1})


def run_euler3d(args):
    """3D Euler 512^3, periodic, ENO-AO7: FP32 bulk vs FP64 (a few steps)."""
    import torch
    import paper_2108_12742_gb300 as eno
    from paper_2108_12742_gb300 import inputs
    clk = ClockSampler(0)
    clk.start()
    win = {}
    n = args.n3d
    U = torch.from_numpy(inputs.euler3d_blast(n, seed=1)).cuda()
    cells = n ** 3
    stream = torch.cuda.current_stream()
    out = {}
    states = {}
    for name, prec, k in (("fp32_bulk", eno.FP32_BULK, args.steps3d), ("fp64", eno.FP64, 1)):
        with eno.Solver((n, n, n), (0.0,) * 3, (1.0,) * 3, stream=stream, system=eno.EULER,
                        order=7, bc=eno.PERIODIC, precision=prec) as s:
            s.init_state(U)
            if not args.no_autotune and prec == eno.FP32_BULK:
                s.autotune()
                s.init_state(U)
            t0 = time.monotonic()
            # three warm-up steps for the FP32-bulk line; one for FP64 (2 s a step)
            ms = _timed_steps(s, k, 3 if prec == eno.FP32_BULK else 1, CFL, stream)
            win[name] = (t0, time.monotonic())
            kms = [s.time_sweep(d, 2) for d in range(3)]
            s.init_state(U)
            s.advance_steps(1, CFL)
            st = torch.empty_like(U)
            s.get_state(st)
            states[name] = st
            out[name] = {"value": cells * 3 * k / (ms / 1e3), "ms_per_step": ms / k, "steps": k,
                         "kernel_ms": kms, "tiles": [s.get_tiles(d) for d in range(3)]}
    diff = (states["fp32_bulk"] - states["fp64"]).abs()
    l1 = [float(diff[v].mean() / states["fp64"][v].abs().mean()) for v in range(5)]
    linf = [float(diff[v].max() / states["fp64"][v].abs().max()) for v in range(5)]
    clocks = clk.stop(*win["fp32_bulk"])
    out["fp64"]["clocks"] = clk.stop(*win["fp64"])
    peaks_run = measure_peaks(0)
    mp, _ = measured_peaks()
    roof = step_roofline(out["fp32_bulk"]["value"], 6000, 107, 347, peaks_run, mp["hbm_gbs"])
    _line(f"euler3d-{n}^3-periodic-blast-ao7", out["fp32_bulk"]["value"],
          out["fp32_bulk"]["ms_per_step"], out["fp32_bulk"]["steps"], 3,
          {"clocks": clocks, "config": {"workload": f"euler3d-{n}^3-periodic-blast-ao7", "cells": cells, "order": 7},
           "fp64": out["fp64"], "kernel_ms_fp32_bulk": out["fp32_bulk"]["kernel_ms"],
           "tiles_fp32_bulk": out["fp32_bulk"].get("tiles"), "roofline": roof,
           "fp32_bulk_speedup_vs_fp64": out["fp32_bulk"]["value"] / out["fp64"]["value"],
           "l1_rel_fp32_bulk_vs_fp64_one_step": l1, "linf_rel_fp32_bulk_vs_fp64_one_step": linf})


def run_small(args, workload):
    """Launch-bound single problems run to their end time: the 1D Euler Riemann
    workload (N = 2000, t_end = 0.2) and the periodic advection (N = 200, t = 2,
    the sine and the seeded square pulse), FP32 bulk and FP64, with the
    FP32-bulk state's L1 / Linf difference from the FP64 one at t_end."""
    import torch
    import paper_2108_12742_gb300 as eno
    from paper_2108_12742_gb300 import inputs
    if workload == "euler1d":
        n, t_end, kw = 2000, 0.2, dict(system=eno.EULER, order=5, bc=eno.TRANSMISSIVE)
        runs = [("riemann-seed1", inputs.euler1d_riemann(n, seed=1))]
        lo, hi = 0.0, 1.0
        name = "euler1d-2000-riemann-ao5-to-t0.2"
    else:
        n, t_end, kw = 200, 2.0, dict(system=eno.SCALAR_ADVECTION, order=5, bc=eno.PERIODIC)
        runs = [("sine", inputs.advection_sine(n)), ("square-seed1", inputs.advection_square(n, 1))]
        lo, hi = -1.0, 1.0
        name = "advection1d-200-sine-and-square-ao5-to-t2"
    clk = ClockSampler(0)
    clk.start()
    results = {}
    for ic, U in runs:
        out, states = {}, {}
        for pname, prec in (("fp32_bulk", eno.FP32_BULK), ("fp64", eno.FP64)):
            with eno.Solver((n,), (lo,), (hi,), precision=prec, **kw) as s:
                s.init_state(U)
                s.advance(t_end, cfl=CFL)       # warm-up run (graph capture)
                s.init_state(U)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                t, k = s.advance(t_end, cfl=CFL)
                sec = time.perf_counter() - t0
                states[pname] = s.get_state()
                out[pname] = {"value": n * 3 * k / sec, "steps": k, "seconds": sec, "t": t}
        a, b = states["fp32_bulk"], states["fp64"]
        nv = a.shape[0]
        out["l1_rel_fp32_bulk_vs_fp64"] = [float(np.abs(a[v] - b[v]).mean() / np.abs(b[v]).mean())
                                           for v in range(nv)]
        out["linf_rel_fp32_bulk_vs_fp64"] = [float(np.abs(a[v] - b[v]).max() / np.abs(b[v]).max())
                                             for v in range(nv)]
        results[ic] = out
    clocks = clk.stop()
    first = results[runs[0][0]]
    _line(name, first["fp32_bulk"]["value"],
          1e3 * first["fp32_bulk"]["seconds"] / first["fp32_bulk"]["steps"],
          first["fp32_bulk"]["steps"], 1,
          {"config": {"workload": name, "cells": n, "cfl": CFL},
           "runs": results, "clocks": clocks,
           "note": "launch-bound: whole run timed on the host clock; value: first run, FP32 bulk"})


def run_convergence(args):
    """The Sec. 4.1 convergence workload on the GPU: u_t + u_x = 0 on [-1, 1],
    periodic, u0 = sin(pi x), t = 2, errors against the exact solution at
    N = 25, 50, 100, 200, 400, FP64: ENO-AO5 at CFL 0.5 (third-order
    Runge-Kutta error dominates: expected order 3) and at dt = dx^(5/3)
    (designed order 5), ENO-AO7 at dt = dx^(7/3) (designed order 7); the
    observed orders log2(e(N) / e(2N))."""
    import paper_2108_12742_gb300 as eno
    from paper_2108_12742_gb300 import inputs
    ns = [25, 50, 100, 200, 400]
    clk = ClockSampler(0)
    clk.start()
    t0 = time.perf_counter()
    cases = {}
    for label, order, dtexp in (("ao5-cfl0.5", 5, None), ("ao5-dt-dx^(5/3)", 5, 5 / 3),
                                ("ao7-dt-dx^(7/3)", 7, 7 / 3)):
        rows = []
        for n in ns:
            U0 = inputs.advection_sine(n)
            dx = 2.0 / n
            with eno.Solver((n,), (-1.0,), (1.0,), system=eno.SCALAR_ADVECTION, order=order,
                            bc=eno.PERIODIC) as s:
                s.init_state(U0)
                if dtexp is None:
                    t, k = s.advance(2.0, cfl=CFL)
                else:
                    t, k = s.advance(2.0, dt_fixed=dx ** dtexp)
                e = np.abs(s.get_state() - U0)   # the exact solution at t = 2 is u0
            rows.append({"n": n, "steps": k, "l1": float(e.mean()), "linf": float(e.max())})
        for i in range(1, len(rows)):
            rows[i]["order_l1"] = float(np.log2(rows[i - 1]["l1"] / rows[i]["l1"]))
            rows[i]["order_linf"] = float(np.log2(rows[i - 1]["linf"] / rows[i]["linf"]))
        cases[label] = rows
    sec = time.perf_counter() - t0
    clocks = clk.stop()
    cells_steps = sum(r["n"] * r["steps"] for rows in cases.values() for r in rows)
    _line("convergence-advection1d-sine-n25-400", cells_steps * 3 / sec, 1e3 * sec, 1, 0,
          {"config": {"workload": "convergence-advection1d-sine-n25-400", "dtype": "f64"},
           "dtype": "f64", "convergence": cases, "clocks": clocks,
           "note": "value: cell-stage updates per host second over all runs (launch-bound)"})


def run_sweep_profile(args):
    """One sweep kernel of a chosen workload, for profiler captures: builds the
    2D four-quadrant data (the benchmark's, at n x n; --ndim 3 the 3D blast at
    n^3; --case riemann2 the 2D Riemann configuration 2 on [-1, 1]^2), takes
    --steps-before steps, sets the tiles and re-decision mode and launches the
    sweep of axis --dir nrep times (enoao_time_sweep), printing the mean."""
    import paper_2108_12742_gb300 as eno
    from paper_2108_12742_gb300 import inputs
    n = args.prof_n
    prec = eno.FP32_BULK if args.prof_precision == "fp32" else eno.FP64
    if args.prof_case == "riemann2":
        U = inputs.riemann2d(2, n, n)
        s = eno.Solver((n, n), (-1.0, -1.0), (1.0, 1.0), system=eno.EULER, order=args.prof_order,
                       bc=eno.TRANSMISSIVE, precision=prec)
    elif args.prof_ndim == 2:
        U = inputs.euler2d_quadrants(n, n, seed=1)
        s = eno.Solver((n, n), (0.0, 0.0), (1.0, 1.0), system=eno.EULER, order=args.prof_order,
                       bc=eno.TRANSMISSIVE, precision=prec)
    else:
        U = inputs.euler3d_blast(n, seed=1)
        s = eno.Solver((n, n, n), (0.0,) * 3, (1.0,) * 3, system=eno.EULER, order=args.prof_order,
                       bc=eno.PERIODIC, precision=prec)
    with s:
        s.set_redecide(eno.REDECIDE_GRID if args.prof_redecide == "grid" else eno.REDECIDE_IN_SWEEP)
        s.init_state(U)
        if args.steps_before:
            s.advance_steps(args.steps_before, CFL)
        if args.prof_ta or args.prof_ts:
            s.set_tiles(args.prof_dir, args.prof_ta, args.prof_ts)
        f0 = s.stats().fp64_fallbacks
        ms = s.time_sweep(args.prof_dir, args.prof_nrep)
        f1 = s.stats().fp64_fallbacks
        print(f"sweep axis {args.prof_dir} {args.prof_precision} n={n} "
              f"tiles={s.get_tiles(args.prof_dir)}: {ms:.4f} ms per launch, "
              f"{(f1 - f0) / (args.prof_nrep + 1):.0f} FP64 re-decisions per launch")
    return 0


def run_paper_cases(args):
    """The paper's printed test cases (Sec. 4) at its resolutions and end times,
    FP32 bulk and FP64 (the 2D cases also FP32 bulk with the grid-wide FP64
    re-decision pass): composite advection wave (dx = 1/200 on [-1, 1], t = 20),
    Lax tube (dx = 1/100 on [0, 2], t = 0.26), Titarev-Toro (dx = 1/200 on
    [-5, 5], t = 5), 2D Riemann configurations 1 and 2 (800 x 800 cells on
    [-1, 1]^2, t = 1); ENO-AO5 and ENO-AO7.  Whole runs timed on the host clock
    (the 1D cases are launch-bound)."""
    import torch
    import paper_2108_12742_gb300 as eno
    from paper_2108_12742_gb300 import inputs
    clk = ClockSampler(0)
    clk.start()
    n2 = args.paper_n2d
    cases = [
        ("composite-wave", inputs.composite_wave(400), (400,), (-1.0,), (1.0,),
         eno.SCALAR_ADVECTION, eno.PERIODIC, 20.0),
        ("lax", inputs.lax_tube(200), (200,), (0.0,), (2.0,), eno.EULER, eno.TRANSMISSIVE, 0.26),
        ("titarev-toro", inputs.titarev_toro(2000), (2000,), (-5.0,), (5.0,), eno.EULER,
         eno.TRANSMISSIVE, 5.0),
        ("riemann2d-1", inputs.riemann2d(1, n2, n2), (n2, n2), (-1.0, -1.0), (1.0, 1.0),
         eno.EULER, eno.TRANSMISSIVE, 1.0),
        ("riemann2d-2", inputs.riemann2d(2, n2, n2), (n2, n2), (-1.0, -1.0), (1.0, 1.0),
         eno.EULER, eno.TRANSMISSIVE, 1.0),
    ]
    rows = []
    total_cs, total_s = 0.0, 0.0
    for name, U, shape, lo, hi, system, bc, t_end in cases:
        cells = int(np.prod(shape))
        for order in (5, 7):
            res = {}
            variants = [("fp32_bulk", eno.FP32_BULK, eno.REDECIDE_AUTO), ("fp64", eno.FP64, eno.REDECIDE_AUTO)]
            if len(shape) > 1:  # shock / slip-line flows: also the grid-wide re-decision pass
                variants.append(("fp32_bulk_grid", eno.FP32_BULK, eno.REDECIDE_GRID))
            for pname, prec, redecide in variants:
                with eno.Solver(shape, lo, hi, system=system, order=order, bc=bc,
                                precision=prec) as s:
                    s.set_redecide(redecide)
                    s.init_state(U)
                    s.advance_steps(1, CFL)     # graph capture outside the timed run
                    s.init_state(U)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    t, k = s.advance(t_end, cfl=CFL)
                    sec = time.perf_counter() - t0
                    res[pname] = (s.get_state(), k, sec, t)
            a, b = res["fp32_bulk"][0], res["fp64"][0]
            row = {"case": name, "order": order, "cells": cells, "t_end": t_end,
                   "steps": res["fp32_bulk"][1],
                   "fp32_bulk_cell_stage_per_s": cells * 3 * res["fp32_bulk"][1] / res["fp32_bulk"][2],
                   "fp64_cell_stage_per_s": cells * 3 * res["fp64"][1] / res["fp64"][2],
                   "fp32_bulk_seconds": res["fp32_bulk"][2], "fp64_seconds": res["fp64"][2],
                   "l1_rel_fp32_bulk_vs_fp64": float(np.abs(a - b).mean() / np.abs(b).mean())}
            if "fp32_bulk_grid" in res:
                g = res["fp32_bulk_grid"]
                row["fp32_bulk_grid_cell_stage_per_s"] = cells * 3 * g[1] / g[2]
                row["fp32_bulk_grid_seconds"] = g[2]
                row["l1_rel_fp32_bulk_grid_vs_fp64"] = float(np.abs(g[0] - b).mean() / np.abs(b).mean())
            if bc == eno.PERIODIC:
                row["conservation_rel_fp64"] = float(abs(b.sum() - U.sum()) / np.abs(U).sum())
            if system == eno.EULER:
                row["min_density_fp64"] = float(b[0].min())
            rows.append(row)
            total_cs += cells * 3 * res["fp32_bulk"][1]
            total_s += res["fp32_bulk"][2]
    clocks = clk.stop()
    _line(f"paper-cases-riemann2d-{n2}", total_cs / total_s, 1e3 * total_s, len(rows), 1,
          {"clocks": clocks, "config": {"workload": f"paper-cases (Sec. 4), 2D at {n2}x{n2}"}, "cases": rows,
           "note": "value: all FP32-bulk runs together, cell-stage updates per host second"})


def run_adr(args):
    """The ADR spectral-analysis tool (Sec. 4.1): modified wavenumbers of
    ENO-AO5 and ENO-AO7 at amplitude 1 for every mode k = 1 .. N/2 of an N-cell
    periodic grid, all modes in one flux sweep; timed end to end on the host
    clock (H2D of the modes, the sweep, D2H of the fluxes, the FFT) and the
    sweep kernel alone with CUDA events."""
    import torch
    import paper_2108_12742_gb300 as eno
    from paper_2108_12742_gb300 import adr
    clk = ClockSampler(0)
    clk.start()
    n = args.adr_n
    out = {}
    for order in (5, 7):
        for pname, prec in (("fp32_bulk", eno.FP32_BULK), ("fp64", eno.FP64)):
            adr.adr(n=256, order=order, precision=prec)  # warm-up (build, first launch)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            theta, kp = adr.adr(n=n, order=order, precision=prec)
            sec = time.perf_counter() - t0
            k, _, U = adr.modes(n)
            with eno.Solver((n, k.size), (0.0, 0.0), (float(n), float(k.size)),
                            system=eno.SCALAR_ADVECTION, order=order, bc=eno.PERIODIC,
                            adv_speed=1.0, precision=prec) as s:
                s.init_state(U)
                kms = s.time_sweep(0, 3)
            out[f"ao{order}_{pname}"] = {"modes_per_s": theta.size / sec, "seconds": sec,
                                         "kernel_ms": kms, "kappa": kp}
    d5 = float(np.abs(out["ao5_fp32_bulk"]["kappa"] - out["ao5_fp64"]["kappa"]).max())
    d7 = float(np.abs(out["ao7_fp32_bulk"]["kappa"] - out["ao7_fp64"]["kappa"]).max())
    for v in out.values():
        del v["kappa"]
    clocks = clk.stop()
    _line(f"adr-{n}-modes", out["ao5_fp64"]["modes_per_s"], 1e3 * out["ao5_fp64"]["seconds"], 1, 1,
          {"clocks": clocks, "config": {"workload": f"ADR of ENO-AO5/AO7, {n // 2} cosine modes of amplitude 1 on "
                                  f"{n} periodic cells, one sweep"},
           "unit": "modes/s", "dtype": "f64",
           "unit_note": "value: ENO-AO5 FP64 modes per host second, end to end",
           "results": out, "max_abs_kappa_fp32_bulk_vs_fp64": {"ao5": d5, "ao7": d7}})


def run_tie_study(args):
    """FP32-bulk near-tie margin study: for each tie_rel, the stencil choices of
    the FP32-bulk path against the FP64 path (itself oracle-identical) on
    evolved 2D four-quadrant data, the FP64 re-decisions per step and the step
    time."""
    import torch
    import paper_2108_12742_gb300 as eno
    from paper_2108_12742_gb300 import inputs
    clk = ClockSampler(0)
    clk.start()
    n, before = args.tie_n, args.tie_evolve
    U = inputs.euler2d_quadrants(n, n, seed=1)
    kw = dict(system=eno.EULER, order=5)
    with eno.Solver((n, n), (0.0, 0.0), (1.0, 1.0), **kw) as s:
        s.init_state(U)
        s.advance_steps(before, 0.5)
        Ue = s.get_state()
        ref = [s.reconstruct_fluxes(d, want_idx=True)[1] for d in range(2)]
    rows = []
    for tr in (1e-2, 1e-3, 1e-4, 1e-5, 0.0):
        with eno.Solver((n, n), (0.0, 0.0), (1.0, 1.0), precision=eno.FP32_BULK, tie_rel=tr,
                        **kw) as s:
            s.init_state(Ue)
            f0 = s.stats().fp64_fallbacks
            dis = tot = 0
            for d in range(2):
                _, idx = s.reconstruct_fluxes(d, want_idx=True)
                dis += int((idx != ref[d]).sum())
                tot += int(idx.size)
            f1 = s.stats().fp64_fallbacks
            s.init_state(Ue)
            s.advance_steps(2, 0.5)
            torch.cuda.synchronize()
            f2 = s.stats().fp64_fallbacks
            t0 = time.perf_counter()
            s.advance_steps(args.steps, 0.5)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / args.steps
            f3 = s.stats().fp64_fallbacks
        rows.append({"tie_rel": tr, "choices": tot, "disagreements": dis,
                     "agreement": 1.0 - dis / tot, "redecided_in_flux_pass": f1 - f0,
                     "redecided_per_step": (f3 - f2) / args.steps, "ms_per_step": ms})
    best = min(rows, key=lambda r: r["ms_per_step"])
    cells = n * n
    clocks = clk.stop()
    _line(f"tie-study-euler2d-{n}x{n}-evolved{before}", cells * 3 / (best["ms_per_step"] * 1e-3),
          best["ms_per_step"], args.steps, 2,
          {"clocks": clocks, "config": {"workload": f"tie-study-euler2d-{n}x{n}-evolved{before}", "order": 5},
           "tie_study": rows,
           "note": "value: fastest tie_rel; agreement against the FP64 path on the same state"})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--cpu-sub", type=int, default=1536)
    ap.add_argument("--cpu-sub1", type=int, default=512)
    ap.add_argument("--agree-sub", type=int, default=384)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tiles", default="",
                    help="FP32-bulk tiles x_lines,x_faces,y_lines,y_faces instead of autotuning")
    ap.add_argument("--workload", default="euler2d",
                    choices=["euler2d", "batched", "euler3d", "euler1d", "advection",
                             "tie-study", "paper-cases", "adr", "convergence", "sweep"])
    # --workload sweep: one sweep kernel (profiler captures)
    ap.add_argument("--prof-n", type=int, default=2048)
    ap.add_argument("--prof-ndim", type=int, default=2, choices=[2, 3])
    ap.add_argument("--prof-order", type=int, default=5)
    ap.add_argument("--prof-precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--prof-dir", type=int, default=0)
    ap.add_argument("--prof-nrep", type=int, default=2)
    ap.add_argument("--prof-ta", type=int, default=0)
    ap.add_argument("--prof-ts", type=int, default=0)
    ap.add_argument("--prof-case", default="quadrants", choices=["quadrants", "riemann2"])
    ap.add_argument("--prof-redecide", default="in_sweep", choices=["in_sweep", "grid"])
    ap.add_argument("--steps-before", type=int, default=0)
    ap.add_argument("--adr-n", type=int, default=4096)
    ap.add_argument("--paper-n2d", type=int, default=800)
    ap.add_argument("--tie-n", type=int, default=2048)
    ap.add_argument("--tie-evolve", type=int, default=200)
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--batch-subset", type=int, default=128)
    ap.add_argument("--n3d", type=int, default=512)
    ap.add_argument("--steps3d", type=int, default=8)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "euler3d":
        return run_euler3d(args)
    if args.workload in ("euler1d", "advection"):
        return run_small(args, args.workload)
    if args.workload == "tie-study":
        return run_tie_study(args)
    if args.workload == "adr":
        return run_adr(args)
    if args.workload == "paper-cases":
        return run_paper_cases(args)
    if args.workload == "convergence":
        return run_convergence(args)
    if args.workload == "sweep":
        return run_sweep_profile(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
