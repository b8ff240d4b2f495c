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

# Algorithmic operations per unit of work of each kernel, counted from the
# formulas (add, sub, mul, min, max, compare = 1; fused multiply-add = 2;
# divide, square root = 1), split by the pipe they run on in each precision.
# The cell-only terms of the half-step prediction (rho div v, grad p / rho,
# gamma p div v: 7 operations) are counted once per cell in k_cell_gradient,
# where they are computed, not once per edge side; the prediction of each
# side is phi + g.(off - hdt u) - hdt src with u = v - wf formed once for
# the shift and the boost (30 operations per side), and HLLC forms the total
# energy of the upwind side only.
# (per unit, unit kind, extra per ring slot)
FLOPS = {
    "fp64": {
        "k_circumcentre": ({"fp64": 24}, "tri", {}),
        "k_edge_geometry": ({"fp64": 32}, "edge", {}),
        "k_cell_geometry": ({"fp64": 27}, "cell", {"fp64": 11}),
        "k_cell_gradient": ({"fp64": 47}, "cell", {"fp64": 83}),
        "k_edge_flux": ({"fp64": 175}, "edge", {}),
        "k_cell_update": ({"fp64": 20}, "cell", {"fp64": 4}),
    },
    "split": {
        "k_circumcentre": ({"fp64": 24}, "tri", {}),
        "k_edge_geometry": ({"fp64": 6, "fp32": 26}, "edge", {}),
        "k_cell_geometry": ({"fp64": 17, "fp32": 10}, "cell", {"fp64": 11}),
        "k_cell_gradient": ({"fp32": 47}, "cell", {"fp32": 83}),
        "k_edge_flux": ({"fp32": 175}, "edge", {}),
        "k_cell_update": ({"fp64": 20}, "cell", {"fp64": 4}),
    },
}


# DRAM bytes (read + write) per unit of the dominant kernel from one ncu
# capture of the kernel version in this tree (profiles/*_sedov262k.md give
# the command and the raw counters), scaled to a launch by its units.  Set
# to None whenever the kernel changes after the capture.
TRAFFIC_PER_UNIT = {
    "fp64": {"k_edge_flux": 146.2},     # profiles/k_edge_flux_fp64_sedov262k.md
    "split": {"k_cell_geometry": 114.1},  # profiles/k_cell_geometry_split_sedov262k.md
}
# The same captures' sm__pipe_fp64_cycles_active (fraction of peak while the
# SMs are active): how busy the bounding pipe is, whatever the op mix.
PIPE_ACTIVE = {
    "fp64": {"k_edge_flux": 0.889},
    "split": {"k_cell_geometry": 0.781},
}


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
    per, kind, slot = FLOPS[prec][name]
    out = {}
    for pipe in ("fp64", "fp32"):
        out[pipe] = per.get(pipe, 0) * units[kind] + slot.get(pipe, 0) * units["slot"]
    return out


def roofline_of(prec, kern_means, units, sweep_ms):
    """Roofline of the dominant kernel: bound by the pipe that carries most
    of its issue time (FP64 issues at 1/64 of the FP32 rate)."""
    dom = max(kern_means, key=kern_means.get)
    fl = kernel_flops(prec, dom, units)
    t64 = fl["fp64"] / (FP64_PEAK_TFLOPS * 1e12)
    t32 = fl["fp32"] / (FP32_PEAK_TFLOPS * 1e12)
    pipe, peak = ("fp64", FP64_PEAK_TFLOPS) if t64 >= t32 else ("fp32", FP32_PEAK_TFLOPS)
    achieved = fl[pipe] / (kern_means[dom] / 1e3) / 1e12
    tot = {"fp64": 0, "fp32": 0}
    for k in FLOPS[prec]:
        f = kernel_flops(prec, k, units)
        tot["fp64"] += f["fp64"]
        tot["fp32"] += f["fp32"]
    hbm, src = hbm_peak()
    cells_per_s = units["cell"] / (sweep_ms / 1e3)
    per_unit = TRAFFIC_PER_UNIT.get(prec, {}).get(dom)
    traffic = per_unit * units[FLOPS[prec][dom][1]] if per_unit is not None else None
    pipe_active = PIPE_ACTIVE.get(prec, {}).get(dom)
    return {"bound": "alu", "pipe": pipe, "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch (ncu DRAM read + write)",
            "pipe_active_ncu": pipe_active,
            "peak_source": ("derived: 152 SMs x 2 FP64 FMA lanes/clk x 2 flop x 2.07 GHz" if pipe == "fp64"
                            else "derived: 152 SMs x 128 FP32 FMA lanes/clk x 2 flop x 2.07 GHz"),
            "sweep_fp64_tflops": tot["fp64"] / (sweep_ms / 1e3) / 1e12,
            "sweep_fp32_tflops": tot["fp32"] / (sweep_ms / 1e3) / 1e12,
            "hbm_frac_compulsory": cells_per_s * COMPULSORY_BYTES_PER_CELL / (hbm * 1e9),
            "hbm_peak_gbs": hbm, "hbm_peak_source": src,
            "kernel_ms": kern_means}


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

    def time_precision(prec, with_clocks, scheme=0):
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
        # ~4 % slow; the Sedov run itself fails after 66 steps, so a copy
        # takes at most 40)
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
        for _ in range(args.steps):
            ms, info, kt = one_step()
            sweep_ms.append(ms)
            tess_ms.append(info["tess_ms"])
            units = {"tri": info["n_tri"], "edge": info["n_edges"], "cell": n, "slot": info["n_slots"]}
            for k, v in kt.items():
                kern.setdefault(k, []).append(v / sweeps_per_step)
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
        means = {k: float(np.mean(v)) for k, v in kern.items() if k != "dt_reset"}
        return {"value": job_value(ws, n * args.steps, total_s), "sweep_ms": sweep_ms, "tess_ms": tess_ms, "wall": wall,
                "units": units, "kernel_means": means, "clocks": clk}

    res64 = time_precision("fp64", True)
    res32 = time_precision("split", False)
    restc = time_precision("fp64", False, scheme=1)
    sweep_ms, tess_ms, wall, units, clk = (res64["sweep_ms"], res64["tess_ms"], res64["wall"], res64["units"],
                                           res64["clocks"])
    value = res64["value"]

    # end to end through the public API: rich_step (host tessellation, copies,
    # sweep) plus a host read of the step's result
    e2e_steps = max(2, min(args.steps, 5))
    bufs = [np.empty(n) for _ in range(6)]
    import ctypes as C
    Dp = C.POINTER(C.c_double)
    L = rich.lib()
    sim2 = rich.Sim(wl)
    sim2.step(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = d2h = 0
    parts = {"tess_ms": 0.0, "copy_ms": 0.0, "sweep_ms": 0.0}
    for _ in range(e2e_steps):
        info = sim2.step(1)
        for k in parts:
            parts[k] += info[k] / e2e_steps
        rc = L.rich_get_conserved(sim2.h, n, *[b.ctypes.data_as(Dp) for b in bufs])
        assert rc == 0
        # what rich_tessellate uploads: ghost positions, sources, mirror
        # flags and shifts; triangles; ring offsets, processing order and
        # first owned edge per cell; ring neighbours and triangles (the
        # edge list itself is built on the device)
        h2d = (28 * info["n_ghost"] + 12 * info["n_tri"] + 4 * (n + 1) + 4 * n + 4 * (n + 1)
               + 8 * info["n_slots"])
        d2h = 16 * n + 12 + 48 * n
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, ws)
    e2e_val = job_value(ws, n * e2e_steps, e2e_s)
    sim2.close()

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    roof = roofline_of("fp64", res64["kernel_means"], units, float(np.mean(sweep_ms)))
    roof32 = roofline_of("split", res32["kernel_means"], res32["units"], float(np.mean(res32["sweep_ms"])))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(sweep_ms)),
        "p50_ms": float(np.percentile(sweep_ms, 50)), "p99_ms": float(np.percentile(sweep_ms, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "cells": n, "precision": "fp64", "scheme": "extrapolated fluxes",
                   "l2": "flushed (256 MB write) before every timed sweep",
                   "warmup": f"{args.warmup} steps, after {args.warmup_seconds:g} s of steps of throwaway copies",
                   "host_tess_ms_per_step": float(np.mean(tess_ms)),
                   "wall_ms_per_step": 1e3 * wall / args.steps, "parallelism": f"replicas x{ws}"},
        "roofline": roof,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "steps": e2e_steps, "ms_per_step": 1e3 * e2e_s / e2e_steps,
                "host_tess_ms": parts["tess_ms"], "copy_ms": parts["copy_ms"], "sweep_ms": parts["sweep_ms"]},
        "gpu_launches": 6 * args.steps,
        "clocks": clk,
        "fp32_split": {"value": res32["value"], "unit": UNIT, "dtype": "f32 reconstruction + f64 geometry/state",
                       "ms_per_step": float(np.mean(res32["sweep_ms"])),
                       "p99_ms": float(np.percentile(res32["sweep_ms"], 99)), "roofline": roof32},
        "time_centred": {"value": restc["value"], "unit": UNIT, "dtype": "f64", "sweeps_per_step": 2,
                         "ms_per_step": float(np.mean(restc["sweep_ms"])),
                         "p99_ms": float(np.percentile(restc["sweep_ms"], 99)),
                         "host_tess_ms_per_step": float(np.mean(restc["tess_ms"])),
                         "kernel_ms_per_sweep": restc["kernel_means"]},
    }
    if not args.no_batched:
        line["batched"] = {"fp64": run_batched(rich, 0, args.batch_instances, args.batch_steps),
                           "fp32_split": run_batched(rich, 1, args.batch_instances, args.batch_steps)}
    if not args.no_serving:
        line["serving"] = run_serving(rich, 1, args.serve_requests, args.serve_steps, 4000, 64000, 0.8)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


def run_batched(rich, precision, n_inst, steps, seed=4):
    """256 independent simulations (sizes log-uniform in 1k-64k, Sod / Sedov /
    Gresho) advanced as one batch: one device sweep per step over all cells.
    The autotuner's 8 trial steps run first (untimed)."""
    from paper_1410_3219_gb300 import workloads as W
    wls = W.batch_mix(n_inst=n_inst, seed=seed)
    b = rich.Batch(precision=precision, max_cells=1 << 26)
    for wl in wls:
        wl["cfg"]["precision"] = precision
        b.add(wl, max_steps=1 << 40)
    cells = sum(len(wl["x"]) for wl in wls)
    for _ in range(8):
        b.step()
    sweep_ms, tess_ms, wall = [], [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        info = b.step()
        wall.append(1e3 * (time.perf_counter() - t0))
        sweep_ms.append(info["sweep_ms"])
        tess_ms.append(info["tess_ms"])
    li = b.launch_info()
    b.close()
    return {"value": cells * steps / (sum(sweep_ms) / 1e3), "unit": UNIT, "instances": n_inst, "cells": cells,
            "ms_per_step": float(np.mean(sweep_ms)), "p99_ms": float(np.percentile(sweep_ms, 99)),
            "host_tess_ms_per_step": float(np.mean(tess_ms)),
            "e2e": {"value": cells * steps / (sum(wall) / 1e3), "unit": UNIT,
                    "wall_ms_per_step": float(np.mean(wall))},
            "launch": {"persistent": li["persistent"], "block": li["block"], "grid": li["grid"],
                       "graph_replay": li["graph"]},
            "gpu_launches_per_step": 1 if li["persistent"] else 6}


def run_serving(rich, precision, n_req, steps_per_req, n_min, n_max, load, seed=5):
    """Requests (Sod / Sedov / Gresho, sizes log-uniform in [n_min, n_max],
    Lloyd eta in [0.01, 0.1], chi in [0.5, 1.5]) served two ways on the same
    GPU: one at a time through rich_step (FIFO), and through the
    continuous-batching server.  Both see the same Poisson arrival stream,
    whose rate is `load` times the one-at-a-time service capacity measured
    first; latency is arrival to result on the host.  Capacity is also
    measured with every request submitted at once."""
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
    total = sum(cells) * steps_per_req

    def solo(wl):
        sim = rich.Sim(wl)
        sim.step(steps_per_req)
        sim.conserved()
        sim.close()

    # one-at-a-time capacity
    t0 = time.perf_counter()
    for wl in reqs:
        solo(wl)
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
        srv = rich.Server(precision=precision, max_cells=1 << 24)
        ids, k = [], 0
        t0 = time.perf_counter()
        sweep_ms = 0.0
        while k < n_req or any(srv.query(r)["state"] in ("queued", "running") for r in ids):
            now = time.perf_counter() - t0
            while k < n_req and arr[k] <= now:
                ids.append(srv.submit(reqs[k], max_steps=steps_per_req))
                k += 1
            if not ids or all(srv.query(r)["state"] in ("done", "failed") for r in ids):
                if k < n_req:
                    time.sleep(max(0.0, arr[k] - (time.perf_counter() - t0)))
                continue
            sweep_ms += srv.tick()["sweep_ms"]
        span = time.perf_counter() - t0
        lat = [srv.query(r)["latency_ms"] for r in ids]
        for r in ids:
            srv.fetch(r)
        srv.close()
        return span, lat, sweep_ms

    span, lat, sweep_ms = serve(arrivals)
    burst_span, _, burst_sweep = serve(np.zeros(n_req))
    return {"requests": n_req, "steps_per_request": steps_per_req, "cells_range": [n_min, n_max],
            "offered_load": load, "unit": UNIT, "latency": "arrival to result on the host",
            "served": {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                       "capacity": total / burst_span, "device_value": total / (burst_sweep / 1e3)},
            "one_at_a_time": {"p50_ms": float(np.percentile(solo_lat, 50)),
                              "p99_ms": float(np.percentile(solo_lat, 99)), "capacity": total / t_solo}}


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
    ap.add_argument("--workload", default="sedov_262144")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--batch-instances", type=int, default=256)
    ap.add_argument("--batch-steps", type=int, default=5)
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-steps", type=int, default=20)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
