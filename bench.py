"""Benchmark of the GB300 PonD time step.

Workload (one bench step = one PonD time step over the whole grid): the 2D
periodic advected Gaussian density/temperature pulse, D2Q16 (f) + D2Q9 (g),
256 x 256 cells, background Mach 2 at 30 degrees, amplitude 0.1, seeded
centre/width, FP64 populations, BGK, dt from CFL 0.2 (1000 steps is the full
run).  Metric: MLUPS = cells x steps / seconds / 1e6.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the context's stream; the L2 cache (129 MB, larger than the 29 MB state)
is flushed by a 256 MiB write between timed steps, outside the events.
``e2e`` repeats the run through the public C ABI with host buffers: pond_init
from pinned host arrays, then per step pond_step(1) + pond_moments into pinned
host arrays, wall-clock timed.

Under torchrun (N > 1) every rank runs an independent replica (the grid is
not sharded; there is no collective on the data path) and ``value`` is the
sum of all ranks' cell updates over the slowest rank's time.

``--impl reference`` times the FP64 CPU oracle instead (each step: one oracle
step on a 64 x 64 window of the same workload) on the host cores.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS per GB300 (FP32 batched vs FP64 plain, stated L1 err); serve p50/p99 latency"
UNIT = "MLUPS"
WORKLOAD = "2D periodic advected Gaussian pulse, D2Q16+D2Q9, 256x256, Mach 2 at 30 deg, FP64, BGK"
# FP64 work of one cell update of the 2D FP64 step (flops, an FMA counting 2):
# 2 DFMA + DADD + DMUL thread instructions per launch / cells, counted by ncu
# on this workload (profiles/step_kernel_fp64_pulse256.md); the analytic count
# per phase is in the design notes.  Bytes one cell update must move: the
# state read once and written once, 28 doubles each way.
FLOPS_PER_CELL_2D_FP64 = 11656.5
BYTES_PER_CELL_2D_FP64 = 2 * 28 * 8
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12  # 2 FP64 FMA/clk/SM at 2070 MHz
# dram__bytes_read.sum + dram__bytes_write.sum of one step-kernel launch, keyed
# by the digest of the CUDA sources it was captured from (null once they change)
TRAFFIC_BY_DIGEST = {
    "4c37b29d0b1e0bed4d0de8fa34da26004ca0587081a332f2530188e9370f89b1": 15382016,
}


def _build_digest():
    from paper_2302_00310_gb300 import build as B

    return B._digest()


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return None, 0, 1
    import torch.distributed as dist

    backend = "nccl"
    dist.init_process_group(backend=backend)
    return dist, dist.get_rank(), ws


def _oracle_rate(cfg, fields, n_window: int, steps: int, budget_s: float | None = None):
    """Oracle MLUPS on an n_window^2 periodic window of the workload."""
    import oracle

    sub = [np.ascontiguousarray(a[:n_window, :n_window]) for a in fields]
    d = dict(cfg, nx=n_window, ny=n_window)
    ocfg = oracle.Config.from_dict(d)
    st = oracle.init(ocfg, *sub)
    done, t0 = 0, time.perf_counter()
    while done < steps:
        st = oracle.run(ocfg, st, 1)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return n_window * n_window * done / el / 1e6, done, el, oracle.threads()


def run_reference(args, rank, ws):
    """The reference arm: the FP64 oracle on the host cores, rank 0 only."""
    if rank != 0:
        return
    from paper_2302_00310_gb300 import workloads as W

    w = W.pulse_2d(n=256, seed=0)
    fields = (w["rho"], w["ux"], w["uy"], w["T"])
    _oracle_rate(w["cfg"], fields, 64, max(1, args.warmup))
    rate, done, el, thr = _oracle_rate(w["cfg"], fields, 64, args.steps)
    sample = "%d oracle steps on a 64x64 periodic window of the 256x256 pulse" % done
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / done,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "cells": 256 * 256},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, dist, rank, ws):
    import torch

    from paper_2302_00310_gb300 import pond
    from paper_2302_00310_gb300 import workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    pond.lib(build=True)
    w = W.pulse_2d(n=256, seed=0)
    cfg = dict(w["cfg"])
    n = cfg["nx"] * cfg["ny"]
    sim = pond.Sim(cfg)
    stream = sim.stream
    sim.init(w["rho"], w["ux"], w["uy"], w["T"])
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # warm-up
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            pond.pond_step(sim.ctx, 1)
    stream.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()  # L2 flush, outside the timed events
                ev[i][0].record(stream)
                pond.pond_step(sim.ctx, 1)
                ev[i][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if dist is not None:
        dist.barrier()
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    sum_ms = float(sum(kernel_ms))
    st, flags, max_cfl, _ = sim.flags()

    # end to end through the C ABI with pinned host buffers
    hin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
           (w["rho"], w["ux"], w["uy"], w["T"])]
    hout = [torch.empty((cfg["ny"], cfg["nx"]), dtype=torch.float64).pin_memory() for _ in range(4)]
    hin_np = [t.numpy() for t in hin]
    hout_np = [t.numpy() for t in hout]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pond.pond_init(sim.ctx, *hin_np)
    for _ in range(args.steps):
        pond.pond_step(sim.ctx, 1)
        pond.pond_moments(sim.ctx, *hout_np)
    e2e_s = time.perf_counter() - t0
    sim.close()

    if dist is not None:
        t = torch.tensor([sum_ms, e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        sum_ms, e2e_s = float(t[0]), float(t[1])
    if rank != 0:
        return
    mlups = n * args.steps * ws / (sum_ms * 1e-3) / 1e6
    e2e = n * args.steps * ws / e2e_s / 1e6
    per_launch_s = sum_ms * 1e-3 / args.steps
    achieved = FLOPS_PER_CELL_2D_FP64 * n / per_launch_s / 1e12
    line = {
        "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "cells": n, "dt": cfg["dt"], "tau": cfg["tau"],
                   "precision": "fp64", "transform": "tensor", "limiter": "vanleer",
                   "l2": "flushed (256 MiB write) between timed steps",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": TRAFFIC_BY_DIGEST.get(_build_digest()),
                     "kernel": "pond::step_kernel<double,2,8,8,160>",
                     "flops_per_cell": FLOPS_PER_CELL_2D_FP64,
                     "peak_source": "FP64: 2 FMA/clk/SM x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s)",
                     "hbm": {"achieved_gbs": BYTES_PER_CELL_2D_FP64 * n / per_launch_s / 1e9,
                             "peak_gbs": _measured_peaks().get("hbm_gbs", 6652.0)}},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 4 * n * 8 / args.steps,
                "d2h_bytes_per_step": 4 * n * 8},
        "gpu_launches": args.steps,
        "status_flags": flags, "max_cfl": max_cfl,
        "wall_s": t_wall,
    }
    line["roofline"]["hbm"]["frac"] = line["roofline"]["hbm"]["achieved_gbs"] / line["roofline"]["hbm"]["peak_gbs"]
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if ws == 1 and not args.no_cpu_baseline:
        rate, done, el, thr = _oracle_rate(cfg, (w["rho"], w["ux"], w["uy"], w["T"]), 256, 30,
                                          budget_s=10.0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
                                "sample": "%d oracle steps of the full 256x256 grid (%.1f s)" % (done, el)}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, rank, int(os.environ.get("WORLD_SIZE", "1")))
        return
    dist, rank, ws = _dist()
    try:
        run_gpu(args, dist, rank, ws)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
