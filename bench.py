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

# FP64 peak derived from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk x
# 2 flop x 2.070 GHz (max SM clock); a throughput probe measured 1.19 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12

# Algorithmic FP64 operations per unit of work of each kernel, counted from
# the formulas (add, sub, mul, min, max = 1; fused multiply-add = 2; divide
# and square root = 1).  Units: triangles, edges or cells.
FLOPS = {
    "k_circumcentre": (24, "tri"),
    "k_edge_geometry": (31, "edge"),
    "k_cell_geometry": (22, "cell"),       # + 12 per ring slot
    "k_cell_gradient": (40, "cell"),       # + 83 per ring slot
    "k_edge_flux": (224, "edge"),
    "k_cell_update": (20, "cell"),         # + 4 per ring slot
}
PER_SLOT = {"k_cell_geometry": 12, "k_cell_gradient": 83, "k_cell_update": 4}


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


def kernel_flops(name, units):
    per, kind = FLOPS[name]
    f = per * units[kind]
    if name in PER_SLOT:
        f += PER_SLOT[name] * units["slot"]
    return f


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
    sim = rich.Sim(wl)
    sim.set_stream(stream.cuda_stream)
    rich.rich_set_profiling(sim.h, True)

    def one_step(timed):
        info = sim.tessellate()
        with torch.cuda.stream(stream):
            flush.zero_()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            sim.sweep()
            ev1.record(stream)
        res = sim.sync()
        ev1.synchronize()
        return ev0.elapsed_time(ev1), info, res

    for _ in range(args.warmup):
        one_step(False)

    clocks = Clocks(os.path.join(ROOT, "gpurun_out", f"bench_clocks_r{rank}.csv")) if rank == 0 else None
    os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
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
        ms, info, res = one_step(True)
        sweep_ms.append(ms)
        tess_ms.append(info["tess_ms"])
        units = {"tri": info["n_tri"], "edge": info["n_edges"], "cell": n, "slot": info["n_slots"]}
        for k, v in rich.rich_kernel_times(sim.h).items():
            kern.setdefault(k, []).append(v)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if ws > 1:
        dist.barrier()
    clk = clocks.stop(local) if clocks else None

    total_sweep_s = sum(sweep_ms) / 1e3
    if ws > 1:
        t = torch.tensor([total_sweep_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_sweep_s = float(t.item())
    value = ws * n * args.steps / total_sweep_s

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
    for _ in range(e2e_steps):
        info = sim2.step(1)
        rc = L.rich_get_conserved(sim2.h, n, *[b.ctypes.data_as(Dp) for b in bufs])
        assert rc == 0
        h2d = (16 * info["n_ghost"] + 8 * info["n_ghost"] + 12 * info["n_tri"] + 4 * (n + 1)
               + 12 * info["n_slots"] + 16 * info["n_edges"])
        d2h = 16 * n + 12 + 48 * n
    e2e_s = time.perf_counter() - t0
    e2e_val = ws * n * e2e_steps / e2e_s
    sim2.close()

    if rank != 0:
        sim.close()
        if ws > 1:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (FP64-ALU bound)
    means = {k: float(np.mean(v)) for k, v in kern.items() if k != "dt_reset"}
    dom = max(means, key=means.get)
    fl = kernel_flops(dom, units)
    achieved = fl / (means[dom] / 1e3) / 1e12
    total_fl = sum(kernel_flops(k, units) for k in FLOPS)
    roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
            "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
            "sweep_fp64_tflops": total_fl / (float(np.mean(sweep_ms)) / 1e3) / 1e12,
            "kernel_ms": means}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(sweep_ms)),
        "p50_ms": float(np.percentile(sweep_ms, 50)), "p99_ms": float(np.percentile(sweep_ms, 99)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "cells": n, "precision": "fp64", "scheme": "extrapolated fluxes",
                   "l2": "flushed (256 MB write) before every timed sweep",
                   "host_tess_ms_per_step": float(np.mean(tess_ms)),
                   "wall_ms_per_step": 1e3 * wall / args.steps, "parallelism": f"replicas x{ws}"},
        "roofline": roof,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "steps": e2e_steps},
        "gpu_launches": 6 * args.steps,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_seconds)
    sim.close()
    print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


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
    ap.add_argument("--workload", default="sedov_262144")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
