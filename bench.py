"""Benchmark of the moving-Voronoi-mesh sweep (cell-updates per second).

One step = the host tessellation (a0, timed separately) followed by the
device sweep a1-a9.  `value` is real cells x steps / summed device time of
the sweeps (CUDA events on the launching stream, inputs resident in HBM, L2
flushed before every timed sweep).  `e2e` is the same metric through the
public C ABI call a user makes (rich_step with the host tessellation and all
host<->device copies, plus a host read of the step's result).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
       python bench.py --impl reference ...   (the CPU oracle, bounded sample)
Under torchrun every rank advances its own independent instance (replicas;
no data exchange) and rank 0 prints the whole-job line.
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

METRIC = "cell-updates/s of Voronoi sweep (FP64 vs FP32-split, batched), % HBM roofline; p99"
UNIT = "cell-updates/s"

# Peaks derived from unit counts and clocks (2.070 GHz max SM clock):
# FP64: 152 SMs x 2 FMA lanes/clk x 2 flop (an FMA probe measured 1.19 TFLOP/s);
# FP32: 152 SMs x 128 FMA lanes/clk x 2 flop (the probe measured 69.6 TFLOP/s).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# HBM: measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), and the
# compulsory traffic of one cell-update with FP64 state and 32-bit indices:
# read points 16 + U 32 + connectivity ~28, write U 32 + points 16 = 124 B.
HBM_PEAK_GBS_FALLBACK = 6800.0
COMPULSORY_BYTES_PER_CELL = 124
# kernels launched by one sweep
NUM_KERNELS = 6

# Algorithmic floating-point operations of each kernel, counted from the
# formulas as the kernels evaluate them: add, subtract, multiply = 1, fused
# multiply-add = 2, divide, square root and reciprocal square root = 1 (the
# extra FMAs that refine a reciprocal are not counted); compares, min/max,
# sign flips and the FP64 <-> FP32 conversions run on the integer pipe and
# are not counted.  Per unit kind (triangle, edge, cell, ring slot) and pipe.
FLOPS = {
    "fp64": {
        "k_circumcentre": {"tri": {"fp64": 25}},
        "k_geometry": {"edge": {"fp64": 32}, "cell": {"fp64": 52}, "slot": {"fp64": 11}},
        "k_advance_points": {"cell": {"fp64": 5}},
        "k_cell_gradient": {"cell": {"fp64": 67}, "slot": {"fp64": 33}},
        "k_edge_flux": {"edge": {"fp64": 177}},
        "k_cell_update": {"cell": {"fp64": 17}, "slot": {"fp64": 4}},
    },
    "split": {
        "k_circumcentre": {"tri": {"fp64": 25}},
        "k_geometry": {"edge": {"fp64": 6, "fp32": 26}, "cell": {"fp64": 24, "fp32": 29}, "slot": {"fp64": 11}},
        "k_advance_points": {"cell": {"fp64": 5}},
        "k_cell_gradient": {"cell": {"fp32": 67}, "slot": {"fp64": 1, "fp32": 32}},
        "k_edge_flux": {"edge": {"fp64": 1, "fp32": 176}},
        "k_cell_update": {"cell": {"fp64": 17}, "slot": {"fp64": 4}},
    },
}


# DRAM traffic and FP64-pipe activity per kernel come from the committed ncu
# summary of the same workload (profiles/sweep_ncu_<workload>.md, which gives
# the command), and only while the kernel sources still hash to the value
# recorded there: after a kernel change they are null until captured again.
KERNEL_SOURCES = ["sweep.cu", "sweep.cuh", "fp64ops.cuh"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1410_3219_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_summary(workload_name):
    """{precision: {kernel: {"dram_bytes": B, "fp64_pipe": f, ...}}} from the
    committed summary, or {} when it is missing or its kernel-source hash is
    not the current one."""
    path = os.path.join(ROOT, "profiles", f"sweep_ncu_{workload_name}.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return {}, None
    import re
    want = kernel_source_hash()
    got = next((re.search(r"`([0-9a-f]+)`", ln) for ln in lines if ln.startswith("kernel-source-hash:")), None)
    got = got.group(1) if got else None
    if got != want:
        return {}, path
    out = {}
    for ln in lines:
        f = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(f) >= 5 and f[0] in ("fp64", "split"):
            try:
                out.setdefault(f[0], {})[f[1]] = {"dram_bytes": float(f[2]), "fp64_pipe": float(f[3]),
                                                  "duration_us": float(f[4]), "fp64_warp_instr": float(f[5])}
            except ValueError:
                continue
    return out, path


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return HBM_PEAK_GBS_FALLBACK, "fallback"


def workload(name):
    from paper_1410_3219_gb300 import workloads as W
    if name == "sedov_262144":
        return W.sedov(n=262144, seed=2)
    if name == "kh_1048576":
        return W.kelvin_helmholtz(n_side=1024, seed=3)
    if name == "kh_262144":  # the same problem at 512^2, for profiler captures
        return W.kelvin_helmholtz(n_side=512, seed=3)
    if name == "sod_4096":
        return W.sod(n_side=64, seed=1)
    raise SystemExit(f"unknown workload {name}")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, device="cuda"):
    """The largest of the ranks' values of x (the job's time is its slowest
    rank's).  Replicas exchange nothing else."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, units_per_rank, seconds):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return ws * units_per_rank / seconds


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, gpu_index=0):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2])); pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "power_w_max": max(pw), "reasons": sorted(reasons)}


def kernel_flops(prec, name, units):
    out = {"fp64": 0, "fp32": 0}
    for kind, per in FLOPS[prec][name].items():
        for pipe, v in per.items():
            out[pipe] += v * units[kind]
    return out


def roofline_of(prec, kern_means, units, sweep_ms, workload_name, probe=None):
    """Roofline of the dominant kernel (the longest launch of the sweep):
    algorithmic operations on the pipe that carries most of its issue time
    (FP64 issues at 1/64 of the FP32 rate) over its CUDA-event mean
    duration, against the peak derived from unit counts and clocks, with
    the measured FMA-chain peak beside it.  DRAM traffic and FP64-pipe
    activity come from the committed ncu summary while the kernel sources
    still match it."""
    dom = max(kern_means, key=kern_means.get)
    fl = kernel_flops(prec, dom, units)
    t64 = fl["fp64"] / (FP64_PEAK_TFLOPS * 1e12)
    t32 = fl["fp32"] / (FP32_PEAK_TFLOPS * 1e12)
    pipe, peak = ("fp64", FP64_PEAK_TFLOPS) if t64 >= t32 else ("fp32", FP32_PEAK_TFLOPS)
    achieved = fl[pipe] / (kern_means[dom] / 1e3) / 1e12
    tot = {"fp64": 0, "fp32": 0}
    per_kernel = {}
    for k in FLOPS[prec]:
        f = kernel_flops(prec, k, units)
        tot["fp64"] += f["fp64"]
        tot["fp32"] += f["fp32"]
        if k in kern_means:
            per_kernel[k] = {"ms": kern_means[k],
                             "fp64_tflops": f["fp64"] / (kern_means[k] / 1e3) / 1e12,
                             "fp64_frac": f["fp64"] / (kern_means[k] / 1e3) / 1e12 / FP64_PEAK_TFLOPS}
    hbm, src = hbm_peak()
    cells_per_s = units["cell"] / (sweep_ms / 1e3)
    summ, summ_path = ncu_summary(workload_name)
    rec = summ.get(prec, {})
    traffic = rec[dom]["dram_bytes"] if dom in rec else None
    pipe_active = rec[dom]["fp64_pipe"] if dom in rec else None
    sweep_dram = sum(v["dram_bytes"] for v in rec.values()) if len(rec) == len(FLOPS[prec]) else None
    # the FP64 issue bound: GB300 issues one FP64 warp-instruction per 16
    # clocks per SM; the instructions a sweep issues (ncu) at that rate
    sweep_fp64_instr = sum(v["fp64_warp_instr"] for v in rec.values()) if len(rec) == len(FLOPS[prec]) else None
    issue_floor_ms = (sweep_fp64_instr * 16 / 152 / 2.07e9 * 1e3) if sweep_fp64_instr else None
    for k, v in rec.items():
        if k in per_kernel:
            per_kernel[k]["dram_bytes_ncu"] = v["dram_bytes"]
            per_kernel[k]["fp64_pipe_active_ncu"] = v["fp64_pipe"]
    out = {"bound": "alu", "pipe": pipe, "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
           "frac": achieved / peak, "traffic": traffic,
           "traffic_unit": "DRAM bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
           "traffic_source": (os.path.relpath(summ_path, ROOT) if traffic is not None else
                              "null: no ncu summary for this kernel-source hash"),
           "kernel_source_hash": kernel_source_hash(),
           "pipe_active_ncu": pipe_active,
           "peak_source": ("derived: 152 SMs x 2 FP64 FMA lanes/clk x 2 flop x 2.07 GHz" if pipe == "fp64"
                           else "derived: 152 SMs x 128 FP32 FMA lanes/clk x 2 flop x 2.07 GHz"),
           "ops_counted": "FP64-pipe (or FP32-pipe) arithmetic only: add, sub, mul = 1, FMA = 2, divide and "
                          "square root = 1; compares, min/max, sign flips and conversions on the integer pipe "
                          "are not counted",
           "sweep_fp64_tflops": tot["fp64"] / (sweep_ms / 1e3) / 1e12,
           "sweep_fp32_tflops": tot["fp32"] / (sweep_ms / 1e3) / 1e12,
           "sweep_dram_bytes_per_step_ncu": sweep_dram,
           "sweep_fp64_warp_instructions_ncu": sweep_fp64_instr,
           "fp64_issue_floor_ms": issue_floor_ms,
           "fp64_issue_frac": (issue_floor_ms / sweep_ms) if issue_floor_ms else None,
           "fp64_issue_note": "the sweep's FP64 warp-instructions (ncu) at one per 16 clocks per SM, 152 SMs, "
                              "2.07 GHz, over the measured sweep time",
           "hbm_frac_compulsory": cells_per_s * COMPULSORY_BYTES_PER_CELL / (hbm * 1e9),
           "hbm_frac_ncu": (sweep_dram / (sweep_ms / 1e3) / (hbm * 1e9)) if sweep_dram else None,
           "hbm_peak_gbs": hbm, "hbm_peak_source": src,
           "kernels": per_kernel}
    if probe:
        pk = probe["fp64"] if pipe == "fp64" else probe["fp32"]
        out["peak_probe"] = pk
        out["frac_of_probe"] = achieved / pk
        out["peak_probe_source"] = "measured: FMA chains on this GPU (rich_probe_pipe_peaks)"
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_1410_3219_gb300 import rich

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    __graft_entry__.build_library()

    wl = workload(args.workload)
    n = len(wl["x"])
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 256 MB > L2
    import tempfile
    clock_dir = tempfile.mkdtemp(prefix="rich_bench_clocks_")

    warm_state = {"done": False}

    def time_precision(wl, prec, with_clocks, scheme=0, steps=None):
        steps = steps or args.steps
        n = len(wl["x"])
        w = dict(wl)
        w["cfg"] = dict(wl["cfg"], precision=1 if prec == "split" else 0, scheme=scheme)
        sim = rich.Sim(w)
        sim.set_stream(stream.cuda_stream)
        # per-stage events only in the extra profiled steps after the timed
        # region: the timed sweeps are bare launches
        prof = {"on": False}
        rich.rich_set_diagnostics(sim.h, False)
        # the time-centred scheme sweeps twice per step (half step, full step)
        sweeps_per_step = 2 if scheme == 1 else 1

        def one_sweep():
            info = sim.tessellate()
            with torch.cuda.stream(stream):
                flush.zero_()
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(stream)
                sim.sweep()
                ev1.record(stream)
            sim.sync()
            ev1.synchronize()
            return ev0.elapsed_time(ev1), info, (rich.rich_kernel_times(sim.h) if prof["on"] else {})

        def one_step():
            ms, tms, kt = 0.0, 0.0, {}
            for _ in range(sweeps_per_step):
                m1, info, k1 = one_sweep()
                ms += m1
                tms += info["tess_ms"]
                for k, v in k1.items():
                    kt[k] = kt.get(k, 0.0) + v
            return ms, dict(info, tess_ms=tms), kt

        # W warm-up steps; before the first timed run, also warmup_seconds
        # of steps of throwaway copies of the run (the steps are mostly host
        # tessellation; on a fresh box the first seconds of FP64 kernels ran
        # ~4 % slow)
        if not warm_state["done"] and args.warmup_seconds > 0:
            t_warm = time.perf_counter()
            while time.perf_counter() - t_warm < args.warmup_seconds:
                spare = rich.Sim(w)
                spare.set_stream(stream.cuda_stream)
                for _ in range(40):
                    if time.perf_counter() - t_warm >= args.warmup_seconds:
                        break
                    spare.tessellate()
                    with torch.cuda.stream(stream):
                        spare.sweep()
                    spare.sync()
                spare.close()
            warm_state["done"] = True
        for _ in range(args.warmup):
            one_step()
        clocks = Clocks(os.path.join(clock_dir, f"clocks_{prec}_r{rank}.csv")) \
            if (rank == 0 and with_clocks) else None
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
            time.sleep(0.3)
        sweep_ms, tess_ms, kern = [], [], {}
        wall0 = time.perf_counter()
        units = None
        for _ in range(steps):
            ms, info, kt = one_step()
            sweep_ms.append(ms)
            tess_ms.append(info["tess_ms"])
            units = {"tri": info["n_tri"], "edge": info["n_edges"], "cell": n, "slot": info["n_slots"]}
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if ws > 1:
            dist.barrier()
        clk = clocks.stop(local) if clocks else None
        # kernel means: three more steps with events between the stages
        rich.rich_set_profiling(sim.h, True)
        prof["on"] = True
        for _ in range(3):
            _, _, kt = one_step()
            for k, v in kt.items():
                kern.setdefault(k, []).append(v / sweeps_per_step)
        sim.close()
        total_s = max_over_ranks(sum(sweep_ms) / 1e3, ws)
        means = {k: float(np.mean(v)) for k, v in kern.items()}
        return {"value": job_value(ws, n * steps, total_s), "sweep_ms": sweep_ms, "tess_ms": tess_ms, "wall": wall,
                "units": units, "kernel_means": means, "clocks": clk, "steps": steps}

    probe = None
    if rank == 0:
        p64, p32 = rich.rich_probe_pipe_peaks()
        probe = {"fp64": p64, "fp32": p32}

    precs = [p.strip() for p in args.precisions.split(",") if p.strip()]
    res = {}
    for k, pr in enumerate(precs):
        if pr == "tc":
            res[pr] = time_precision(wl, "fp64", k == 0, scheme=1)
        else:
            res[pr] = time_precision(wl, pr, k == 0)
    head = res[precs[0]]
    sweep_ms, tess_ms, wall, units, clk = (head["sweep_ms"], head["tess_ms"], head["wall"], head["units"],
                                           head["clocks"])
    value = head["value"]
    head_prec = "split" if precs[0] == "split" else "fp64"

    # end to end through the public API: rich_step (host tessellation, copies,
    # sweep) plus a host read of the step's result
    # (the same K timed steps after the same W warm-up steps as the device
    # measurement, each a whole step with its copies)
    e2e_steps = max(2, args.steps)
    bufs = [np.empty(n) for _ in range(6)]
    import ctypes as C
    Dp = C.POINTER(C.c_double)
    L = rich.lib()
    w_e2e = dict(wl)
    w_e2e["cfg"] = dict(wl["cfg"], precision=1 if head_prec == "split" else 0)
    sim2 = rich.Sim(w_e2e)
    for _ in range(max(1, args.warmup)):
        sim2.step(1)
        L.rich_get_conserved(sim2.h, n, *[b.ctypes.data_as(Dp) for b in bufs])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = d2h = 0
    parts = {"tess_ms": 0.0, "copy_ms": 0.0, "sweep_ms": 0.0}
    phases = {}
    for _ in range(e2e_steps):
        info = sim2.step(1)
        for k in parts:
            parts[k] += info[k] / e2e_steps
        for k, v in rich.rich_tess_phases(sim2.h).items():
            phases[k] = phases.get(k, 0.0) + v / e2e_steps
        rc = L.rich_get_conserved(sim2.h, n, *[b.ctypes.data_as(Dp) for b in bufs])
        assert rc == 0
        # what rich_tessellate uploads: ghost positions, sources, mirror
        # flags and shifts; ring offsets, processing order, first owned
        # edge and first owned triangle per cell; ring neighbours (the
        # triangle and edge lists themselves are built on the device)
        h2d = (28 * info["n_ghost"] + 4 * (n + 1) + 4 * n + 4 * (n + 1) + 4 * (n + 1)
               + 4 * info["n_slots"])
        # down: the moved points and dt read early, the mesh builds' two
        # check flags, the step's dt and status, the conserved state read
        d2h = (16 * n + 8) + 8 + 12 + 48 * n
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, ws)
    e2e_val = job_value(ws, n * e2e_steps, e2e_s)
    sim2.close()

    sedov = None
    if not args.no_sedov and args.workload != "sedov_262144":
        swl = workload("sedov_262144")
        sedov = {}
        for pr in ("fp64", "split"):
            r = time_precision(swl, pr, False)
            sedov[pr] = {"value": r["value"], "unit": UNIT, "ms_per_step": float(np.mean(r["sweep_ms"])),
                         "p99_ms": float(np.percentile(r["sweep_ms"], 99)),
                         "host_tess_ms_per_step": float(np.mean(r["tess_ms"])),
                         "roofline": roofline_of(pr, r["kernel_means"], r["units"], float(np.mean(r["sweep_ms"])),
                                                 "sedov_262144", probe)}

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    roof = roofline_of(head_prec, head["kernel_means"], units, float(np.mean(sweep_ms)), args.workload, probe)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(sweep_ms)),
        "p50_ms": float(np.percentile(sweep_ms, 50)), "p99_ms": float(np.percentile(sweep_ms, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head_prec == "fp64" else "f32 reconstruction + f64 geometry/state",
        "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "cells": n, "precision": head_prec,
                   "scheme": "time-centred fluxes" if precs[0] == "tc" else "extrapolated fluxes",
                   "l2": "flushed (256 MB write) before every timed sweep",
                   "warmup": f"{args.warmup} steps, after {args.warmup_seconds:g} s of steps of throwaway copies",
                   "host_tess_ms_per_step": float(np.mean(tess_ms)),
                   "wall_ms_per_step": 1e3 * wall / args.steps, "parallelism": f"replicas x{ws}"},
        "roofline": roof,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "steps": e2e_steps, "ms_per_step": 1e3 * e2e_s / e2e_steps,
                "host_tess_ms": parts["tess_ms"], "host_tess_phases_ms": phases, "copy_ms": parts["copy_ms"],
                "sweep_ms": parts["sweep_ms"]},
        "gpu_launches": NUM_KERNELS * args.steps * (2 if precs[0] == "tc" else 1),
        "clocks": clk,
        "pipe_peaks_probe_tflops": probe,
    }
    if "split" in res and precs[0] != "split":
        r = res["split"]
        line["fp32_split"] = {"value": r["value"], "unit": UNIT, "dtype": "f32 reconstruction + f64 geometry/state",
                              "ms_per_step": float(np.mean(r["sweep_ms"])),
                              "p99_ms": float(np.percentile(r["sweep_ms"], 99)),
                              "roofline": roofline_of("split", r["kernel_means"], r["units"],
                                                      float(np.mean(r["sweep_ms"])), args.workload, probe)}
    if "tc" in res and precs[0] != "tc":
        r = res["tc"]
        line["time_centred"] = {"value": r["value"], "unit": UNIT, "dtype": "f64", "sweeps_per_step": 2,
                                "ms_per_step": float(np.mean(r["sweep_ms"])),
                                "p99_ms": float(np.percentile(r["sweep_ms"], 99)),
                                "host_tess_ms_per_step": float(np.mean(r["tess_ms"])),
                                "kernel_ms_per_sweep": r["kernel_means"]}
    if sedov:
        line["sedov_262144"] = sedov
    if not args.no_batched:
        line["batched"] = {"fp64": run_batched(rich, 0, args.batch_instances, args.batch_steps),
                           "fp32_split": run_batched(rich, 1, args.batch_instances, args.batch_steps)}
    if not args.no_serving:
        line["serving"] = run_serving(rich, 1, args.serve_requests, args.serve_steps, 4000, 1 << 20, 0.8)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def run_batched(rich, precision, n_inst, steps, seed=4):
    """256 independent simulations (sizes log-uniform in 1k-64k, Sod / Sedov /
    Gresho) advanced as one batch: one device sweep per step over all cells.
    The autotuner's 8 trial steps and 2 more run first (untimed)."""
    from paper_1410_3219_gb300 import workloads as W
    wls = W.batch_mix(n_inst=n_inst, seed=seed)
    b = rich.Batch(precision=precision, max_cells=1 << 26)
    for wl in wls:
        wl["cfg"]["precision"] = precision
        b.add(wl, max_steps=1 << 40)
    cells = sum(len(wl["x"]) for wl in wls)
    # the autotuner's 8 trial steps, then 2 steps in the chosen shape (the
    # first of them tessellates twice: its own points, which the persistent
    # trials left unmeshed, and the next step's during its sweep)
    for _ in range(8 + 2):
        b.step()
    sweep_ms, tess_ms, copy_ms, wall = [], [], [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        info = b.step()
        wall.append(1e3 * (time.perf_counter() - t0))
        sweep_ms.append(info["sweep_ms"])
        tess_ms.append(info["tess_ms"])
        copy_ms.append(info["copy_ms"])
    li = b.launch_info()
    # both launch shapes timed on the same batch, the autotuner's choice first
    shapes = {}
    for name, mode, block in (("staged", 1, 256), ("persistent_256", 2, 256), ("persistent_512", 2, 512)):
        b.set_launch(mode, block)
        b.step()  # records the graph of this shape
        shapes[name] = float(np.mean([b.step()["sweep_ms"] for _ in range(3)]))
    b.close()
    return {"value": cells * steps / (sum(sweep_ms) / 1e3), "unit": UNIT, "instances": n_inst, "cells": cells,
            "shape_ms_per_step": shapes,
            "ms_per_step": float(np.mean(sweep_ms)), "p99_ms": float(np.percentile(sweep_ms, 99)),
            "host_tess_ms_per_step": float(np.mean(tess_ms)),
            "host_other_ms_per_step": float(np.mean(copy_ms)),
            "e2e": {"value": cells * steps / (sum(wall) / 1e3), "unit": UNIT,
                    "wall_ms_per_step": float(np.mean(wall))},
            # (host tessellation + other host work + device sweep) / wall: above
            # 1 where the host's tessellation of the next step runs beside the
            # sweep's last stages
            "host_device_overlap": float((np.mean(tess_ms) + np.mean(copy_ms) + np.mean(sweep_ms)) / np.mean(wall)),
            "launch": {"persistent": li["persistent"], "block": li["block"], "grid": li["grid"],
                       "graph_replay": li["graph"]},
            "gpu_launches_per_step": 1 if li["persistent"] else NUM_KERNELS}


def run_serving(rich, precision, n_req, steps_per_req, n_min, n_max, load, seed=5, lanes=2, split=65536,
                max_cells=1 << 22, top_lane_cells=1 << 20):
    """Requests (Sod / Sedov / Gresho, sizes log-uniform in [n_min, n_max],
    Lloyd eta in [0.01, 0.1], chi in [0.5, 1.5], steps_per_req steps each)
    served two ways on the same GPU: one at a time through rich_step (FIFO),
    and through the continuous-batching server running `lanes` lane threads
    (requests of at least `split` cells in the second lane).  Both see the
    same Poisson arrival stream, whose rate is `load` times the one-at-a-time
    service capacity measured first; latency is arrival to result on the
    host.  Capacity is also measured with every request submitted at once."""
    import math
    from paper_1410_3219_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n_req):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        side = max(4, int(round(math.sqrt(n))))
        kind = k % 3
        eta, chi = float(rng.uniform(0.01, 0.1)), float(rng.uniform(0.5, 1.5))
        if kind == 0:
            wl = W.sod(n_side=side, seed=2000 + k)
        elif kind == 1:
            wl = W.sedov(n=n, seed=2000 + k)
        else:
            wl = W.gresho(n_side=side, seed=2000 + k)
        wl["cfg"].update(eta=eta, chi=chi, precision=precision)
        reqs.append(wl)
    cells = [len(w["x"]) for w in reqs]

    def solo(wl):
        # one step per call, so that a run the scheme stops (a Sedov blast
        # emptying a cell) still counts the steps it made
        sim = rich.Sim(wl)
        done = 0
        try:
            for _ in range(steps_per_req):
                sim.step(1)
                done += 1
        except rich.RichError:
            pass
        sim.conserved()
        sim.close()
        return done

    # one-at-a-time capacity (cell-updates actually done, failed runs included)
    t0 = time.perf_counter()
    solo_updates = 0
    for wl in reqs:
        solo_updates += len(wl["x"]) * solo(wl)
    t_solo = time.perf_counter() - t0
    rate = load * n_req / t_solo
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))

    # one at a time, FIFO, under the arrival stream
    solo_lat = []
    t0 = time.perf_counter()
    for k, wl in enumerate(reqs):
        wait = arrivals[k] - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        solo(wl)
        solo_lat.append(1e3 * (time.perf_counter() - t0 - arrivals[k]))

    def serve(arr):
        srv = rich.Server(precision=precision, max_cells=max_cells)
        srv.start(lanes=lanes, split_cells=split, top_lane_cells=top_lane_cells)
        ids, k = [], 0
        t0 = time.perf_counter()
        while k < n_req:
            now = time.perf_counter() - t0
            while k < n_req and arr[k] <= now:
                ids.append(srv.submit(reqs[k], max_steps=steps_per_req))
                k += 1
            if k < n_req:
                time.sleep(max(0.0, min(0.002, arr[k] - (time.perf_counter() - t0))))
        while any(srv.query(r)["state"] in ("queued", "running") for r in ids):
            time.sleep(0.002)
        span = time.perf_counter() - t0
        lat = [srv.query(r)["latency_ms"] for r in ids]
        updates = sum(c * srv.query(r)["steps"] for c, r in zip(cells, ids))
        st = srv.stats()
        for r in ids:
            srv.fetch(r)
        srv.close()
        return span, lat, updates, st

    span, lat, updates, st = serve(arrivals)
    burst_span, _, burst_updates, bst = serve(np.zeros(n_req))
    return {"requests": n_req, "steps_per_request": steps_per_req, "cells_range": [n_min, n_max],
            "cells_total": int(sum(cells)), "eta_range": [0.01, 0.1], "chi_range": [0.5, 1.5],
            "kinds": "Sod / Sedov / Gresho in turn (Sedov requests stop where the scheme empties a cell)",
            "offered_load": load, "unit": UNIT, "latency": "arrival to result on the host",
            "served": {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                       "value": updates / span, "capacity": burst_updates / burst_span,
                       "device_value": burst_updates / (bst["sweep_ms"] / 1e3) if bst["sweep_ms"] else None,
                       "lanes": lanes, "lane_split_cells": split, "top_lane_cells": top_lane_cells,
                       "budget_cells": max_cells,
                       "burst_device_busy": bst["sweep_ms"] / bst["wall_ms"] if bst["wall_ms"] else None,
                       "burst_host_tess_busy": bst["tess_ms"] / bst["wall_ms"] if bst["wall_ms"] else None,
                       "burst_lane_steps": bst["steps"]},
            "one_at_a_time": {"p50_ms": float(np.percentile(solo_lat, 50)),
                              "p99_ms": float(np.percentile(solo_lat, 99)), "capacity": solo_updates / t_solo}}


def cpu_baseline(wl, budget_s):
    """The oracle as it stands (single thread, FP64) on a bounded sample of
    the same workload: whole sweeps of all cells, tessellation untimed."""
    from oracle import oracle as O
    O.build()
    n = len(wl["x"])
    sim = O.Sim(wl)
    sweeps, spent = 0, 0.0
    while spent < budget_s and sweeps < 20:
        if sweeps:
            sim.tessellate()
        t0 = time.perf_counter()
        sim.sweep()
        spent += time.perf_counter() - t0
        sweeps += 1
    sim.close()
    return {"value": n * sweeps / spent, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sweeps} full sweep(s) of {n} cells (tessellation untimed)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    wl = workload(args.workload)
    from oracle import oracle as O
    O.build()
    n = len(wl["x"])
    sim = O.Sim(wl)
    for _ in range(args.warmup):
        sim.step()
    times = []
    for _ in range(args.steps):
        sim.tessellate()
        t0 = time.perf_counter()
        sim.sweep()
        times.append(time.perf_counter() - t0)
    sim.close()
    value = n * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": {"workload": args.workload, "cells": n, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} full sweeps of {n} cells (tessellation untimed)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--warmup-seconds", type=float, default=3.0)
    ap.add_argument("--workload", default="kh_1048576")
    ap.add_argument("--precisions", default="fp64,split,tc",
                    help="comma list of the sweeps to time: fp64, split, tc (time-centred); the first is the headline")
    ap.add_argument("--no-sedov", action="store_true", help="skip the extra Sedov 262,144-cell lines")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-steps", type=int, default=100)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
