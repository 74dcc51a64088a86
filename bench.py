"""Benchmark of the GB300 PonD time step.

Main line (``value``): the 2D periodic advected Gaussian density/temperature
pulse, D2Q16 (f) + D2Q9 (g), 256 x 256 cells, background Mach 2 at 30 deg,
amplitude 0.1, seeded centre/width, FP64, BGK, dt from CFL 0.2: one bench
step = one PonD time step of the grid (1000 make the full run).  Metric:
MLUPS = cells x steps / seconds / 1e6.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events
on the context's stream; the L2 cache (129 MB, larger than the 29 MB state)
is flushed between timed steps, outside the events: a 256 MiB buffer is
written and another 256 MiB buffer read (so the step also does not pay for
the write-back of the flush's dirty lines).
``e2e`` repeats the run through the public C ABI with host buffers: pond_init
from pinned host arrays, then per step pond_step(1) + pond_moments into
pinned host arrays, wall-clock timed.

The other forms the metric compares are measured in the same run
(``--no-extras`` skips them):
  * ``mixed``: the same pulse on the mixed path (FP32 + FP64 moments), with
    the L1 / Linf relative density error against the FP64 path after the
    full 1000-step run;
  * ``riemann``: the four-quadrant Riemann problem at 1024^2 (QE Pr 0.71),
    mixed path and FP64, with the L1 error between them after 200 steps;
  * ``d2q25``: the pulse on the D2Q25 f-lattice, FP64 and mixed;
  * ``batched``: 64 shock-bubble instances of seeded sizes 64^2-512^2 (about
    4.07M cells), Mach 1.5-5, Pr 0.71, advanced by the persistent batch
    kernel (autotuned), FP32-mixed and FP64, with the L1 error of the mixed
    batch against the FP64 batch after 100 steps;
  * ``serve``: 200 requests of the serving mix (1D tubes and 2D shock-bubble
    problems, Poisson arrivals at 3 requests/s) through the continuous-batching
    server, p50/p99 time to solution and aggregate MLUPS;
  * ``serve_offered``: the same mix offered at 200 requests/s for 30 s of
    wall time: throughput, the latency of the finished requests, the queue;
  * ``iterated``: the iterated face frame against the averaged one on the Sod
    tube and the pulse at CFL 0.2 / 0.5 / 0.8 and two resolutions: L1 errors
    against the exact solutions, traces per face, MLUPS;
  * ``couette``: thermal Couette flow between walls at the paper's size for
    three Prandtl and three Eckert numbers, against the analytic profile;
  * ``serve_sweep``: the serving mix at 1-4 requests/s (50 requests each),
    the sustained rate.

Under torchrun (N > 1) every rank runs an independent replica (the grid is
not sharded; there is no collective on the data path) and ``value`` is the
sum of all ranks' cell updates over the slowest rank's time.  The extras are
single-GPU measurements and run at N = 1 only.

``--impl reference`` times the FP64 CPU oracle instead (each step: one oracle
step on a 64 x 64 window of the same workload) on the host cores.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS per GB300 (FP32 batched vs FP64 plain, stated L1 err); serve p50/p99 latency"
UNIT = "MLUPS"
WORKLOAD = "2D periodic advected Gaussian pulse, D2Q16+D2Q9, 256x256, Mach 2 at 30 deg, FP64, BGK"
# ncu counters of one main-line step launch, keyed by the digest of the step
# kernels' sources and flags they were taken on (build.kernel_digest;
# profiles/ holds the captures; a changed kernel gives None): executed flops per cell update (2 FMA + ADD + MUL
# thread instructions, packed FP32 pairs twice that, per launch / cells) and
# dram__bytes_read.sum + dram__bytes_write.sum per launch.
NCU_BY_DIGEST = {
    "f1e612ccf8a9dc80f4cbd68501088a8ce05ddb6576c3fc724f94647b9c8a59e0": {
        "flops_fp64": 7726.9, "traffic_fp64": 15132288, "flops_fp32": 7780.5, "traffic_fp32": 9575680,
        # the capped mixed tile (code 11) on the 1024^2 Riemann problem, 6th step
        "flops_fp32_riemann": 7599.1, "traffic_fp32_riemann": 280381184},
}


def formulation_flops(qf=4, qg=3, mixed=False):
    """Floating-point operations of one owned 2D cell update in the
    dimensional-Hermite formulation of the step (the algorithmic work: one
    x-face and one y-face per cell, the cell's own update, its phi_bar^+;
    no face computed twice, no non-arithmetic instruction): a fused
    multiply-add counts 2, an add, multiply, division or square root 1.
    Main line: f on D2Q16 (qf = 4 nodes per axis), g on D2Q9 (qg = 3), tensor
    transformation, van Leer, main flux form, BGK, averaged face frame, no
    node at v_n = 0.  mixed: the FP32 work of the mixed path (the face's
    conserved fluxes added; the cell's FP64 moment sums are not FP32 work).

    Per axis and Q-vector: frame change 6 fma (Q = 4) / 3 fma (Q = 3);
    synthesis at the face nodes 8 / 4 fma; analysis 16 / 9 flops;
    multiplication by v 13 / 9 flops (+ 2 / 1 hoisted).  A frame change's
    constants: 9 flops per axis + 2 shared (dT, 3 dT).  Per face and lattice:
    the two cells beside the face in full, the pairs (2, 3), (4, 5), (6, 7)
    with both cells' normal stage and one tangential stage, and per node a
    normal and a tangential limited slope (16 flops, the quotient counted 1).
    """
    def shift(q):
        return {4: 12, 3: 6}[q]

    def synth(q):
        return {4: 16, 3: 8}[q]

    def transform(q, cells):  # tensor-product moves + synthesis of `cells` stencil cells
        return cells * (20 + 2 * q * (shift(q) + synth(q)))

    def pair(q):  # normal stage of both cells, tangential stage once (selected)
        return 40 + 2 * q * (shift(q) + synth(q)) + q * (shift(q) + synth(q))

    def trace(q):
        setup = {4: 6, 3: 2}[q] + 3 + 7 * q              # synthesis constants, offsets per node
        return setup + transform(q, 2) + 3 * pair(q) + q * q * 16

    ana = {4: 7 + 8 * 16, 3: 3 + 6 * 9}
    face = 8 + trace(qf) + trace(qg) + ana[qf] + ana[qg] + 15      # frame, traces, analysis, moments
    face += 1 + 12 + 3 + sum(q - 1 + q + 2 * q * (q - 1) for q in (qf, qg))  # closed-form equilibrium
    if mixed:
        face += 20                                                   # conserved fluxes of the face
    vmul = {4: 4 * 13 + 2, 3: 3 * 9 + 1}
    move_to_cell = 20 + 2 * qf * shift(qf) + 2 * qg * shift(qg)     # one face's phi into the cell frame
    per_dir = 2 * move_to_cell + (qf * qf + qg * qg) + vmul[qf] + vmul[qg] + 2 * (qf * qf + qg * qg)
    cell = (qf * qf + qg * qg) + 2 * per_dir + 6 + 15 + (2 + 18 + 2 * qf * shift(qf) + 2 * qg * shift(qg)) + 3
    prep = (qf * qf + qg * qg) + 5
    return 2 * face + cell + prep


BYTES_PER_CELL_FP64 = 2 * 28 * 8          # state read once + written once
BYTES_PER_CELL_FP32 = 2 * (28 * 4 + 4 * 8)  # + the FP64 conserved moments
CLOCK_MAX_GHZ = 2.07
# nominal unit-count peaks (context only: the roofline divides by the FMA
# peaks that pond_measure_fma_peak() measures in the same run)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * CLOCK_MAX_GHZ / 1e3     # 2 FP64 FMA/clk/SM
FP32_PEAK_TFLOPS = 152 * 128 * 2 * CLOCK_MAX_GHZ / 1e3   # 128 FP32 FMA/clk/SM
# the step kernels the main line launches, as the profiler names them
KERNEL_FP64 = "member_step_kernel<double, 2, 4, 8, 14, 128, 2, 0, 0, 3>"
KERNEL_FP32 = "member_step_kernel<float, 2, 4, 8, 14, 128, 2, 0, 0, 3>"
# the mixed path's kernel on grids of at least four waves of three CTAs per SM
KERNEL_FP32_CAPPED = "member_step_kernel<float, 2, 4, 8, 14, 128, 3, 0, 0, 3>"


def _build_digest():
    from paper_2302_00310_gb300 import build as B

    return B.kernel_digest()


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

    dist.init_process_group(backend="nccl")
    return dist, dist.get_rank(), ws


def _max_over_ranks(dist, values, device):
    """Element-wise maximum of per-rank timings over all ranks (the slowest
    rank sets the job's time); identity without a process group."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def _job_rate(cells: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job MLUPS: every rank advances its own replica of `cells` cells by
    `steps` steps; the job takes the slowest rank's `seconds`."""
    return cells * steps * world / seconds / 1e6


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


def _time_steps(torch, pond, sim, steps, flush=None):
    """Per-step CUDA-event times (ms) of `steps` single steps on the context
    stream.  flush: a pair of device buffers larger than L2; before each timed
    step the first is written and the second read, so that the step starts
    with a cold and clean L2 (the write alone would leave dirty lines whose
    write-back lands inside the timed step)."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    stream = sim.stream
    with torch.cuda.stream(stream):
        for i in range(steps):
            if flush is not None:
                flush[0].zero_()  # L2 flush, outside the timed events
                flush[2].copy_(flush[1].sum(dtype=torch.int64))
            ev[i][0].record(stream)
            pond.pond_step(sim.ctx, 1)
            ev[i][1].record(stream)
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def _l1(a, b):
    return float(np.sum(np.abs(a - b)) / np.sum(np.abs(b)))


def _linf(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _roofline(key, cells, per_launch_s, peak, bytes_per_cell, kernel, digest, ncu_key=None,
              flops_note=""):
    """ALU roofline of one step launch: the formulation's flops of an owned
    cell update (formulation_flops) times the cells of a launch over the
    launch's CUDA-event time, against `peak` (TFLOP/s and how it was
    obtained); the kernel's executed flops (ncu, with the edge faces two tiles
    share and every helper instruction) and the DRAM traffic beside them, and
    the HBM fraction of the algorithmic bytes.  `ncu_key` names the counters
    of another workload than the main line's (default: `key`)."""
    fpc = formulation_flops(mixed=(key == "fp32"))
    hbm_peak = _measured_peaks().get("hbm_gbs", 6652.0)
    ncu = NCU_BY_DIGEST.get(digest, {})
    nk = ncu_key or key
    out = {"bound": "alu", "unit": "TFLOP/s", "peak": peak["tflops"],
           "peak_source": peak["source"], "kernel": kernel,
           "flops_per_cell": fpc, "flops_source": "formulation count per owned cell update "
                                                  "(bench.formulation_flops)" + flops_note,
           "executed_flops_per_cell": ncu.get("flops_" + nk),
           "achieved": fpc * cells / per_launch_s / 1e12, "frac": None,
           "traffic": ncu.get("traffic_" + nk),
           "hbm": {"achieved_gbs": bytes_per_cell * cells / per_launch_s / 1e9, "peak_gbs": hbm_peak,
                   "bytes_per_cell": bytes_per_cell}}
    out["frac"] = out["achieved"] / peak["tflops"]
    out["hbm"]["frac"] = out["hbm"]["achieved_gbs"] / hbm_peak
    if out["executed_flops_per_cell"]:
        out["executed_tflops"] = out["executed_flops_per_cell"] * cells / per_launch_s / 1e12
    return out


def measure_fma_peaks(pond, local):
    """FP64 and FP32 fma throughput of this GPU (pond_measure_fma_peak), with
    the SM clock sampled while it runs."""
    with ClockSampler(local) as clk:
        fp64, ms64 = pond.pond_measure_fma_peak(pond.POND_FP64, 0.5)
        fp32, ms32 = pond.pond_measure_fma_peak(pond.POND_FP32_MIXED, 0.5)
    out = {"fp64_tflops": fp64, "fp32_tflops": fp32, "launch_ms": {"fp64": ms64, "fp32": ms32},
           "how": "pond_measure_fma_peak: independent fma chains, all SMs, best of 5 launches"}
    c = clk.summary()
    if c:
        out["clocks"] = c
    return out


def _peak(peaks, key):
    src = "measured: pond_measure_fma_peak %s fma chains in this run" % key.upper()
    if c := peaks.get("clocks"):
        src += " at %.0f MHz median SM clock" % c["sm_mhz"]
    return {"tflops": peaks["%s_tflops" % key], "source": src}


def bench_mixed(torch, pond, W, flush, peaks):
    """The pulse on the mixed path: MLUPS and the error of the full run."""
    w = W.pulse_2d(n=256, seed=0)
    fields = (w["rho"], w["ux"], w["uy"], w["T"])
    n = w["cfg"]["nx"] * w["cfg"]["ny"]
    sim = pond.Sim(dict(w["cfg"], precision=pond.POND_FP32_MIXED))
    sim.init(*fields)
    _time_steps(torch, pond, sim, 5)
    ms = _time_steps(torch, pond, sim, 200, flush)
    sim.init(*fields)
    sim.step(w["steps"])
    m32 = sim.moments()
    fl32 = sim.flags()[1]
    tile = sim.info()[2]
    sim.close()
    ref = pond.Sim(w["cfg"])
    ref.init(*fields)
    ref.step(w["steps"])
    m64 = ref.moments()
    ref.close()
    per = sum(ms) / len(ms) * 1e-3
    return {
        "workload": "256x256 pulse as the main line, POND_FP32_MIXED, tile %d" % tile,
        "value": n / per / 1e6, "unit": UNIT, "ms_per_step": per * 1e3,
        "l1_rho_vs_fp64": _l1(m32[0], m64[0]), "linf_rho_vs_fp64": _linf(m32[0], m64[0]),
        "l1_T_vs_fp64": _l1(m32[3], m64[3]), "error_after_steps": w["steps"],
        "mass_drift": float(m32[0].sum() / m64[0].sum() - 1.0), "nonphysical": bool(fl32 & 1),
        "stated_l1_bound": 1e-6,
        "roofline": _roofline("fp32", n, per, _peak(peaks, "fp32"), BYTES_PER_CELL_FP32, KERNEL_FP32,
                              _build_digest()),
    }


def bench_riemann(torch, pond, W, steps=200, peaks=None):
    """The four-quadrant Riemann problem at 1024^2 (seeded states, QE Pr 0.71,
    minmod), mixed path and plain FP64: MLUPS and the L1 error after `steps`;
    with `peaks`, the mixed kernel's roofline (its capped three-CTA tile on
    this grid)."""
    w = W.riemann4_2d(n=1024, seed=1)
    fields = (w["rho"], w["ux"], w["uy"], w["T"])
    n = w["cfg"]["nx"] * w["cfg"]["ny"]
    out = {"workload": "four-quadrant Riemann problem, D2Q16+D2Q9, 1024x1024, seed 1 (quadrant states "
                       "rho in [0.1,1.5], p in [0.03,1.5], Mach up to 3), QE Pr 0.71, minmod, tau 1e-4",
           "cells": n, "steps": steps, "unit": UNIT}
    mom = {}
    for prec, name in ((pond.POND_FP32_MIXED, "fp32_mixed"), (pond.POND_FP64, "fp64")):
        sim = pond.Sim(dict(w["cfg"], precision=prec))
        sim.init(*fields)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(sim.stream):
            e0.record(sim.stream)
            pond.pond_step(sim.ctx, steps)
            e1.record(sim.stream)
        sim.stream.synchronize()
        ms = e0.elapsed_time(e1)
        mom[name] = sim.moments()
        fl = sim.flags()[1]
        tile = sim.info()[2]
        out[name] = {"value": n * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                     "tile": tile, "nonphysical": bool(fl & 1)}
        if peaks is not None and prec == pond.POND_FP32_MIXED:
            out[name]["roofline"] = _roofline(
                "fp32", n, ms * 1e-3 / steps, _peak(peaks, "fp32"), BYTES_PER_CELL_FP32,
                KERNEL_FP32_CAPPED if tile == 11 else KERNEL_FP32, _build_digest(),
                ncu_key="fp32_riemann" if tile == 11 else "fp32_none",
                flops_note="; the main line's count (van Leer, BGK): this problem runs minmod and QE")
        sim.close()
    out["l1_rho_fp32_vs_fp64"] = _l1(mom["fp32_mixed"][0], mom["fp64"][0])
    out["linf_rho_fp32_vs_fp64"] = _linf(mom["fp32_mixed"][0], mom["fp64"][0])
    out["stated_l1_bound"] = 1e-7
    return out


def bench_d2q25(torch, pond, W, steps=100):
    """The D2Q25 f-lattice on the 256^2 pulse (FP64 and mixed), against the
    D2Q16 run of the same workload and dt: MLUPS of both, timed alike, and
    the L1 density difference."""
    w = W.pulse_2d(n=256, seed=0)
    fields = (w["rho"], w["ux"], w["uy"], w["T"])
    n = w["cfg"]["nx"] * w["cfg"]["ny"]
    dt = W.dt_from_cfl(w["ux"], w["uy"], w["T"], w["cfg"]["dx"], 0.2, c_max=W.C_MAX_D1Q5)
    out = {"workload": "256x256 pulse as the main line, D2Q25 f + D2Q9 g, dt from CFL 0.2 on D2Q25's "
                       "nodes", "steps": steps, "unit": UNIT}
    rho = {}
    for qf in (5, 4):
        for prec, name in ((pond.POND_FP64, "fp64"), (pond.POND_FP32_MIXED, "fp32_mixed")):
            sim = pond.Sim(dict(w["cfg"], qf=qf, dt=dt, precision=prec))
            sim.init(*fields)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(sim.stream):
                pond.pond_step(sim.ctx, 3)
                e0.record(sim.stream)
                pond.pond_step(sim.ctx, steps)
                e1.record(sim.stream)
            sim.stream.synchronize()
            ms = e0.elapsed_time(e1)
            rho[(qf, name)] = sim.moments()[0]
            rate = {"value": n * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps, "tile": sim.info()[2]}
            if qf == 5:
                out[name] = rate
            else:
                out.setdefault("d2q16_same_dt", {})[name] = rate
            sim.close()
    out["l1_rho_d2q25_vs_d2q16_fp64"] = _l1(rho[(5, "fp64")], rho[(4, "fp64")])
    out["l1_rho_fp32_vs_fp64_d2q25"] = _l1(rho[(5, "fp32_mixed")], rho[(5, "fp64")])
    out["stated_l1_bound_fp32_vs_fp64"] = 3e-7
    return out


def bench_multiscale(torch, pond, W, steps=200, theta=0.05):
    """The multiscale f-lattice (D2Q9 where smooth, D2Q16 where a velocity or
    temperature jump across a cell exceeds `theta`): the four-quadrant Riemann
    problem at 1024^2 (BGK) in FP64 against plain D2Q16, and the Lax tube of
    Sec. V.C.1 at the paper's L = 600 against its exact solution for D1Q4,
    D1Q3 (every cell low) and the multiscale run."""
    from tests.riemann_exact import solution

    w = W.riemann4_2d(n=1024, seed=1, prandtl=1.0)
    fields = (w["rho"], w["ux"], w["uy"], w["T"])
    n = w["cfg"]["nx"] * w["cfg"]["ny"]
    out = {"workload": "four-quadrant Riemann problem 1024x1024 as the riemann line but BGK (Pr 1), FP64; "
                       "Lax tube L = 600 to t = 0.14", "theta_u": theta, "theta_T": theta,
           "cells": n, "steps": steps, "unit": UNIT}
    mom = {}
    for name, extra in (("d2q16", {}), ("multiscale", dict(ms=1, ms_theta_u=theta, ms_theta_T=theta))):
        sim = pond.Sim(dict(w["cfg"], **extra))
        sim.init(*fields)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(sim.stream):
            e0.record(sim.stream)
            pond.pond_step(sim.ctx, steps)
            e1.record(sim.stream)
        sim.stream.synchronize()
        ms = e0.elapsed_time(e1)
        mom[name] = sim.moments()
        out[name] = {"value": n * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                     "tile": sim.info()[2], "nonphysical": bool(sim.flags()[1] & 1)}
        if extra:
            out[name]["high_fraction"] = sim.ms_stats() / (n * steps)
        sim.close()
    out["l1_rho_multiscale_vs_d2q16"] = _l1(mom["multiscale"][0], mom["d2q16"][0])
    # the mixed path with the main flux form (a low cell's energy flux in its own frame)
    sim = pond.Sim(dict(w["cfg"], precision=pond.POND_FP32_MIXED, ms=1, ms_theta_u=theta, ms_theta_T=theta))
    sim.init(*fields)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(sim.stream):
        e0.record(sim.stream)
        pond.pond_step(sim.ctx, steps)
        e1.record(sim.stream)
    sim.stream.synchronize()
    ms = e0.elapsed_time(e1)
    rho32 = sim.moments()[0]
    out["multiscale_fp32_mixed"] = {"value": n * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                                    "tile": sim.info()[2], "high_fraction": sim.ms_stats() / (n * steps),
                                    "nonphysical": bool(sim.flags()[1] & 1)}
    sim.close()
    out["l1_rho_multiscale_fp32_vs_fp64"] = _l1(rho32, mom["multiscale"][0])
    out["stated_l1_bound_multiscale_fp32_vs_fp64"] = 1e-7
    # the mixed path runs the multiscale lattice in Appendix C's flux form: both precisions in it,
    # beside the mixed D2Q16 kernel in the same form
    appc = {}
    for name, prec, ms_on in (("fp64", pond.POND_FP64, 1), ("fp32_mixed", pond.POND_FP32_MIXED, 1),
                              ("fp32_mixed_d2q16", pond.POND_FP32_MIXED, 0)):
        extra = dict(ms=1, ms_theta_u=theta, ms_theta_T=theta) if ms_on else {}
        sim = pond.Sim(dict(w["cfg"], flux_appc=1, precision=prec, **extra))
        sim.init(*fields)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(sim.stream):
            e0.record(sim.stream)
            pond.pond_step(sim.ctx, steps)
            e1.record(sim.stream)
        sim.stream.synchronize()
        ms = e0.elapsed_time(e1)
        appc[name] = sim.moments()
        out["appc_" + name] = {"value": n * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                               "tile": sim.info()[2], "high_fraction": sim.ms_stats() / (n * steps),
                               "nonphysical": bool(sim.flags()[1] & 1)}
        sim.close()
    out["l1_rho_appc_multiscale_fp32_vs_fp64"] = _l1(appc["fp32_mixed"][0], appc["fp64"][0])
    out["stated_l1_bound_appc_fp32_vs_fp64"] = 1e-7
    left, right = (0.445, 0.698, 3.528), (0.5, 0.0, 0.571)
    lax = W.lax_1d(n=600)
    exact = solution(left, right, lax["x"], lax["t_end"])[0]
    out["lax"] = {"n": 600, "steps": lax["steps"]}
    for name, extra in (("d1q4", {}), ("d1q3", dict(ms=1, ms_theta_u=1e30, ms_theta_T=1e30)),
                        ("multiscale", dict(ms=1, ms_theta_u=theta, ms_theta_T=theta))):
        sim = pond.Sim(dict(lax["cfg"], **extra))
        sim.init(lax["rho"], lax["ux"], lax["uy"], lax["T"])
        sim.step(lax["steps"])
        rho = np.asarray(sim.moments()[0]).ravel()
        out["lax"][name] = {"l1_rho_vs_exact": float(np.mean(np.abs(rho - exact)))}
        if name == "multiscale":
            out["lax"][name]["high_fraction"] = sim.ms_stats() / (600 * lax["steps"])
        sim.close()
    return out


def bench_g_lattice(torch, pond, W, steps=100):
    """The g-populations on the f-lattice (D2Q16 for g) on the 256^2 pulse,
    FP64 and mixed, beside g on D2Q9: MLUPS of both, timed alike, and the L1
    density difference."""
    w = W.pulse_2d(n=256, seed=0)
    fields = (w["rho"], w["ux"], w["uy"], w["T"])
    n = w["cfg"]["nx"] * w["cfg"]["ny"]
    out = {"workload": "the main line's 256x256 pulse, g on D2Q16 against g on D2Q9", "steps": steps,
           "unit": UNIT}
    rho = {}
    for qg in (4, 3):
        for prec, name in ((pond.POND_FP64, "fp64"), (pond.POND_FP32_MIXED, "fp32_mixed")):
            sim = pond.Sim(dict(w["cfg"], qg=qg, precision=prec))
            sim.init(*fields)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(sim.stream):
                pond.pond_step(sim.ctx, 3)
                e0.record(sim.stream)
                pond.pond_step(sim.ctx, steps)
                e1.record(sim.stream)
            sim.stream.synchronize()
            ms = e0.elapsed_time(e1)
            rho[(qg, name)] = sim.moments()[0]
            out.setdefault("g_d2q16" if qg == 4 else "g_d2q9", {})[name] = {
                "value": n * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps, "tile": sim.info()[2]}
            sim.close()
    out["l1_rho_g_d2q16_vs_g_d2q9_fp64"] = _l1(rho[(4, "fp64")], rho[(3, "fp64")])
    out["l1_rho_fp32_vs_fp64_g_d2q16"] = _l1(rho[(4, "fp32_mixed")], rho[(4, "fp64")])
    out["stated_l1_bound_fp32_vs_fp64"] = 3e-7
    return out


def bench_batched(torch, pond, W):
    """64 shock-bubble instances through the persistent batch kernel."""
    ws_ = [W.shock_bubble_2d(seed=s) for s in range(64)]
    cells = sum(w["cfg"]["nx"] * w["cfg"]["ny"] for w in ws_)
    out = {"workload": "64 shock-bubble instances, sides %d-%d (log-uniform seeded), Mach 1.5-5, "
                       "bubble density ratio 0.1-10, Pr 0.71, minmod, tau 1e-3, inflow left" %
                       (min(w["cfg"]["nx"] for w in ws_), max(w["cfg"]["nx"] for w in ws_)),
           "instances": len(ws_), "cells": cells, "unit": UNIT}
    moments = {}
    for prec, name, steps in ((pond.POND_FP32_MIXED, "fp32_mixed", 100), (pond.POND_FP64, "fp64", 20)):
        tune = pond.pond_tune_default()
        tune.graph_steps = 8
        b = pond.Batch(2, prec, len(ws_), tune)
        sims = []
        for w in ws_:
            s = pond.Sim(dict(w["cfg"], precision=prec), stream=b.stream)
            s.init(w["rho"], w["ux"], w["uy"], w["T"])
            b.add(s)
            sims.append(s)
        b.step([24] * len(ws_))       # the autotuner's chunks (3 shapes x 8 steps)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(b.stream)
        b.step([steps] * len(ws_))
        e1.record(b.stream)
        b.stream.synchronize()
        ms = e0.elapsed_time(e1)
        tile, grid, tuned, _ = b.info()
        b.step([200 - 24 - steps] * len(ws_))   # to step 200 for the error statement
        b.stream.synchronize()
        moments[name] = [s.moments()[0] for s in sims]
        nonphys = sum(1 for s in sims if s.flags()[1] & 1)
        b.close()
        for s in sims:
            s.close()
        out[name] = {"value": cells * steps / (ms * 1e-3) / 1e6, "ms_per_step": ms / steps,
                     "tile": tile, "grid": grid, "autotuned": tuned, "nonphysical": nonphys,
                     "timed_steps": steps}
    num = sum(float(np.sum(np.abs(a - b))) for a, b in zip(moments["fp32_mixed"], moments["fp64"]))
    den = sum(float(np.sum(np.abs(b))) for b in moments["fp64"])
    out["l1_rho_fp32_vs_fp64"] = num / den
    out["error_after_steps"] = 200
    out["stated_l1_bound"] = 3e-7
    out["speedup_fp32_batched_vs_fp64"] = out["fp32_mixed"]["value"] / out["fp64"]["value"]
    return out


def bench_iterated(torch, pond, W, iter_tol=1e-9, iter_max=40):
    """The iterated face frame against the averaged one (the comparison of
    Sec. V.D, on problems with exact solutions): Sod tubes and the advected
    pulse at CFL 0.2 / 0.5 / 0.8 and two resolutions, L1 density errors
    against the exact solutions, and the iteration statistics."""
    from tests.riemann_exact import solution

    rows = []
    for n in (100, 400):
        for cfl in (0.2, 0.5, 0.8):
            w = W.sod_1d(n=n, cfl=cfl)
            exact = solution((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), w["x"], w["t_end"])[0]
            row = {"problem": "sod", "n": n, "cfl": cfl, "steps": w["steps"]}
            for it in (0, 1):
                cfg = dict(w["cfg"], iterative=it, iter_tol=iter_tol, iter_max=iter_max)
                sim = pond.Sim(cfg)
                sim.init(w["rho"], w["ux"], w["uy"], w["T"])
                sim.step(w["steps"])
                rho = sim.moments()[0][0]
                ev, tr, mx = sim.iter_stats()
                fl = sim.flags()
                sim.close()
                key = "iterated" if it else "averaged"
                row[key] = {"l1_rho": float(np.sum(np.abs(rho - exact)) / n), "max_cfl": fl[2]}
                if it:
                    row[key].update({"traces_per_face": tr / ev, "max_traces": mx,
                                     "unconverged_frac": fl[3] / ev})
            rows.append(row)
    for n in (64, 128):
        for cfl in (0.2, 0.5, 0.8):
            w = W.pulse_2d(n=n, seed=0, cfl=cfl)
            t_end = 0.25
            steps = int(np.ceil(t_end / w["cfg"]["dt"]))
            cfg0 = dict(w["cfg"], dt=t_end / steps)
            exact = W.pulse_exact_2d(w, t_end)
            row = {"problem": "pulse", "n": n, "cfl": cfl, "steps": steps}
            for it in (0, 1):
                cfg = dict(cfg0, iterative=it, iter_tol=iter_tol, iter_max=iter_max)
                sim = pond.Sim(cfg)
                sim.init(w["rho"], w["ux"], w["uy"], w["T"])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(sim.stream):
                    e0.record(sim.stream)
                    pond.pond_step(sim.ctx, steps)
                    e1.record(sim.stream)
                sim.stream.synchronize()
                ms = e0.elapsed_time(e1)
                rho = sim.moments()[0]
                ev, tr, mx = sim.iter_stats()
                fl = sim.flags()
                sim.close()
                key = "iterated" if it else "averaged"
                row[key] = {"l1_rho_rel": float(np.sum(np.abs(rho - exact)) / np.sum(exact - 1.0)),
                            "mlups": n * n * steps / (ms * 1e-3) / 1e6}
                if it:
                    row[key].update({"traces_per_face": tr / ev, "max_traces": mx,
                                     "unconverged_frac": fl[3] / ev})
            rows.append(row)
    return {"workload": "Sod tube (n = 100, 400; t = 0.2) and the Mach-2 pulse (n = 64, 128; "
                        "t = 0.25), FP64, averaged vs iterated face frame (iter_tol %g, "
                        "iter_max %d)" % (iter_tol, iter_max), "cases": rows}


def bench_couette(torch, pond, W, ny=150, viscous_times=0.25):
    """Thermal Couette flow (Sec. V.B.2) at the paper's parameters (L = 150
    cells, Ma 0.5, Re 100, T_C = 1), Pr 0.5 / 0.7 / 1 x Ec 4 / 20 / 40, FP64,
    walls with the Chapman-Enskog ghost non-equilibrium: the nine runs advance
    together in one batch from the analytic steady state for a quarter of the
    viscous time L^2/nu; the error of the temperature profile against
    (T - T_C)/(T_H - T_C) = y + Pr Ec/2 y (1 - y)."""
    cases = [(pr, ec) for pr in (0.5, 0.7, 1.0) for ec in (4.0, 20.0, 40.0)]
    ws_ = [W.thermal_couette_2d(ny=ny, nx=8, prandtl=pr, ec=ec, re=100.0) for pr, ec in cases]
    steps = [int(viscous_times * (100.0 / w["u0"]) / w["cfg"]["dt"]) for w in ws_]
    tune = pond.pond_tune_default()
    tune.autotune = 0
    b = pond.Batch(2, pond.POND_FP64, len(ws_), tune)
    sims = []
    for w in ws_:
        sim = pond.Sim(w["cfg"], stream=b.stream)
        sim.init(w["rho"], w["ux"], w["uy"], w["T"])
        b.add(sim)
        sims.append(sim)
    t0 = time.perf_counter()
    b.step(steps)
    b.stream.synchronize()
    el = time.perf_counter() - t0
    rows = []
    for (pr, ec), w, sim, n in zip(cases, ws_, sims, steps):
        m = sim.moments()
        theta = (m[3][:, 3] - w["t_cold"]) / w["dT"]
        exact = w["theta"](w["y"])
        rows.append({"prandtl": pr, "eckert": ec, "steps": n,
                     "theta_err_rel": float(np.max(np.abs(theta - exact)) / np.max(exact)),
                     "theta_mid": float(theta[ny // 2]), "theta_mid_exact": float(exact[ny // 2]),
                     "u_err": float(np.max(np.abs(m[1][:, 3] / w["u0"] - w["y"]))),
                     "nonphysical": bool(sim.flags()[1] & 1)})
    b.close()
    for sim in sims:
        sim.close()
    return {"workload": "thermal Couette, 8 x %d cells, Ma 0.5, Re 100, T_C = 1, FP64, nine runs in "
                        "one batch" % ny, "seconds": el, "cases": rows}


def bench_serve(pond, serve_mod, n_requests=200, rate=3.0):
    """The serving statement: a fixed count of requests of the C5 mix at a
    sustainable rate, p50/p99 time to solution over all of them.  The mix
    offers about rate x 3.4e8 cell updates per second (half the requests 2D,
    E[n^2] = 2.5e5 cells, E[steps] = 2750), so 3 requests/s keeps the mixed
    path (about 1.2e9 per second) below saturation; the offered 200/s is far
    beyond one GPU (bench_serve_offered)."""
    reqs = serve_mod.make_requests(n_requests, rate=rate, seed=0)
    ex = serve_mod.PondExecutor(precision=pond.POND_FP32_MIXED, capacity=64, graph_steps=8)
    srv = serve_mod.Server(ex, budget_bytes=16 << 30, tick_steps=64)
    out = srv.run(reqs)
    tile_2d = ex.batches[2].info()[0]
    ex.close()
    s = serve_mod.summary(out)
    s.update({"workload": "Poisson stream at %g req/s: D1Q4 Sod-type tubes (256-8192 cells) and "
                          "D2Q16 shock-bubble runs (128^2-1024^2), 500-5000 steps each, FP32-mixed"
                          % rate,
              "sample": "%d requests (%d 2D), every one finished" % (
                  n_requests, sum(1 for r in out if r.dim == 2)),
              "rate": rate, "budget_gb": 16 << 30 >> 30, "peak_resident_gb": srv.peak_bytes / 1e9,
              "ticks": srv.ticks, "tick_steps": 64, "tile_2d_at_end": tile_2d})
    return s


def bench_serve_offered(pond, serve_mod, n_requests=400, rate=200.0, wall_s=30.0):
    """The C5 stream at its offered 200 requests/s, served for a fixed wall
    time: throughput, the latency of the requests finished by then, and the
    queue left at the end."""
    reqs = serve_mod.make_requests(n_requests, rate=rate, seed=2)
    ex = serve_mod.PondExecutor(precision=pond.POND_FP32_MIXED, capacity=64, graph_steps=8)
    srv = serve_mod.Server(ex, budget_bytes=16 << 30, tick_steps=64)
    out = srv.run(reqs, wall_limit=wall_s)
    tile_2d = ex.batches[2].info()[0]
    ex.close()
    s = serve_mod.summary(out, makespan=srv.stopped_at)
    s.update({"workload": "the C5 mix offered at %g req/s (%d requests drawn), served for %g s of "
                          "wall time, FP32-mixed" % (rate, n_requests, wall_s),
              "wall_limit_s": wall_s, "stopped_at_s": srv.stopped_at, "tile_2d_at_end": tile_2d,
              "note": "p50/p99 over the requests finished within the wall time; the rest are "
                      "counted as running, queued or not yet arrived"})
    return s


def bench_serve_sweep(pond, serve_mod, rates=(1.0, 2.0, 3.0, 4.0), n_requests=50):
    """The C5 stream at lower rates: the offered 200 requests/s is far beyond
    one GPU, so the fixed-count run above measures queueing; this sweep finds
    the rate the server sustains (p99 time to solution within twice its value
    at the lowest rate)."""
    rows = []
    for rate in rates:
        reqs = serve_mod.make_requests(n_requests, rate=rate, seed=1)
        ex = serve_mod.PondExecutor(precision=pond.POND_FP32_MIXED, capacity=64, graph_steps=8)
        srv = serve_mod.Server(ex, budget_bytes=16 << 30, tick_steps=64)
        out = srv.run(reqs)
        ex.close()
        s_ = serve_mod.summary(out)
        rows.append({"rate": rate, "p50_s": s_["p50_s"], "p99_s": s_["p99_s"], "mlups": s_["mlups"],
                     "done": s_["done"]})
    base = rows[0]["p99_s"]
    ok = [r["rate"] for r in rows if r["p99_s"] is not None and r["p99_s"] <= 2.0 * base]
    return {"workload": "the serving stream's request mix, %d requests per rate, FP32-mixed" % n_requests,
            "rates": rows, "sustained_rate": max(ok) if ok else None,
            "criterion": "p99 time to solution <= 2x its value at %g req/s" % rates[0]}


def run_gpu(args, dist, rank, ws):
    import torch

    from paper_2302_00310_gb300 import pond
    from paper_2302_00310_gb300 import serve as serve_mod
    from paper_2302_00310_gb300 import workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    pond.lib(build=True)
    if args.extra:
        if rank == 0 and args.extra == "serve":
            res = {"serve": bench_serve(pond, serve_mod), "serve_offered": bench_serve_offered(pond, serve_mod),
                   "serve_sweep": bench_serve_sweep(pond, serve_mod)}
            print(json.dumps(dict(extra=args.extra, **res)), flush=True)
        elif rank == 0 and args.extra == "riemann":
            res = bench_riemann(torch, pond, W, peaks=measure_fma_peaks(pond, local))
            print(json.dumps(dict(extra=args.extra, **res)), flush=True)
        elif rank == 0:
            fn = {"d2q25": bench_d2q25, "multiscale": bench_multiscale,
                  "g_lattice": bench_g_lattice}[args.extra]
            print(json.dumps(dict(extra=args.extra, **fn(torch, pond, W))), flush=True)
        return
    peaks = measure_fma_peaks(pond, local)
    w = W.pulse_2d(n=256, seed=0)
    fp32 = args.precision == "fp32"
    cfg = dict(w["cfg"], precision=pond.POND_FP32_MIXED if fp32 else pond.POND_FP64)
    n = cfg["nx"] * cfg["ny"]
    sim = pond.Sim(cfg)
    sim.init(w["rho"], w["ux"], w["uy"], w["T"])
    tile = sim.info()[2]
    flush = (torch.empty(256 << 20, dtype=torch.uint8, device="cuda"),
             torch.zeros(256 << 20, dtype=torch.uint8, device="cuda"),
             torch.zeros((), dtype=torch.int64, device="cuda"))
    _time_steps(torch, pond, sim, args.warmup)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        kernel_ms = _time_steps(torch, pond, sim, args.steps, flush)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if dist is not None:
        dist.barrier()
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

    # the extras are single-GPU measurements: at N > 1 they would hold every
    # GPU (the other ranks wait in the reduction below) for minutes
    extras = {}
    if not args.no_extras and ws == 1:
        extras["mixed"] = bench_mixed(torch, pond, W, flush, peaks)
        extras["riemann"] = bench_riemann(torch, pond, W, peaks=peaks)
        extras["batched"] = bench_batched(torch, pond, W)
        extras["d2q25"] = bench_d2q25(torch, pond, W)
        extras["multiscale"] = bench_multiscale(torch, pond, W)
        extras["g_lattice"] = bench_g_lattice(torch, pond, W)
        extras["serve"] = bench_serve(pond, serve_mod)
        extras["serve_offered"] = bench_serve_offered(pond, serve_mod)
        if not args.no_studies:
            extras["serve_sweep"] = bench_serve_sweep(pond, serve_mod)
            extras["iterated"] = bench_iterated(torch, pond, W)
            extras["couette"] = bench_couette(torch, pond, W)

    sum_ms, e2e_s = _max_over_ranks(dist, [sum_ms, e2e_s], "cuda")
    if rank != 0:
        return
    mlups = _job_rate(n, args.steps, ws, sum_ms * 1e-3)
    e2e = _job_rate(n, args.steps, ws, e2e_s)
    per_launch_s = sum_ms * 1e-3 / args.steps
    digest = _build_digest()
    if fp32:
        roof = _roofline("fp32", n, per_launch_s, _peak(peaks, "fp32"), BYTES_PER_CELL_FP32, KERNEL_FP32,
                         digest)
    else:
        roof = _roofline("fp64", n, per_launch_s, _peak(peaks, "fp64"), BYTES_PER_CELL_FP64, KERNEL_FP64,
                         digest)
    line = {
        "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("FP64", "FP32-mixed") if fp32 else WORKLOAD,
                   "cells": n, "dt": cfg["dt"], "tau": cfg["tau"],
                   "precision": args.precision, "transform": "tensor", "limiter": "vanleer",
                   "tile": tile, "l2": "flushed between timed steps (256 MiB written, then another 256 MiB read)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": roof,
        "fma_peaks": peaks,
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 4 * n * 8 / args.steps,
                "d2h_bytes_per_step": 4 * n * 8},
        "gpu_launches": args.steps,
        "status_flags": flags, "max_cfl": max_cfl,
        "wall_s": t_wall,
    }
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    line.update(extras)
    if ws == 1 and not args.no_cpu_baseline:
        import oracle

        rate, done, el, thr = _oracle_rate(cfg, (w["rho"], w["ux"], w["uy"], w["T"]), 256, 30,
                                          budget_s=10.0)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
                                "sample": "%d oracle steps of the full 256x256 grid (%.1f s)" % (done, el)}
        # the same source on one thread (a 64x64 window of the grid, bounded)
        oracle.set_threads(1)
        rate1, done1, el1, _ = _oracle_rate(cfg, (w["rho"], w["ux"], w["uy"], w["T"]), 64, 30,
                                            budget_s=5.0)
        oracle.set_threads(thr)
        line["cpu_baseline"]["single_thread"] = {
            "value": rate1, "unit": UNIT, "cores": 1,
            "sample": "%d oracle steps of a 64x64 window (%.1f s)" % (done1, el1)}
        # the oracle's operation count of one step on the same 64x64 window: the work of the
        # paper's population-space route, beside the kernel's executed flops per cell
        sub = [np.ascontiguousarray(x[:64, :64]) for x in (w["rho"], w["ux"], w["uy"], w["T"])]
        ocfg = oracle.Config.from_dict(dict(cfg, nx=64, ny=64))
        ops, _ = oracle.count_ops(ocfg, oracle.init(ocfg, *sub), 1)
        line["cpu_baseline"]["oracle_ops_per_cell_update"] = ops / (64 * 64)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="main line only (no mixed, batched or served measurements)")
    ap.add_argument("--no-studies", action="store_true",
                    help="skip the accuracy studies (iterated face frame, thermal Couette)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"],
                    help="arithmetic of the main line (fp32 = the mixed path)")
    ap.add_argument("--extra", default=None, choices=["riemann", "d2q25", "multiscale", "g_lattice", "serve"],
                    help="run only this one extra measurement and print its JSON line (for profiling)")
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
