"""Continuous-batching service of PonD simulations on one GPU.

Requests (a 1D tube or a 2D problem with its initial fields and a number of
steps) arrive over time.  The server keeps every admitted request's state
resident on the device, admits queued requests first-come first-served as
soon as their device workspace fits the memory budget, and advances all
admitted requests together: 1D and 2D requests are members of two
``pond_batch`` objects on separate CUDA streams (their work overlaps on the
GPU), each tick advancing every member by up to ``tick_steps`` steps through
the persistent step kernel.  A request whose steps are done is read back
(moments to the host), leaves its batch and frees its memory, and the queue
is admitted again; requests that arrive while others run join at the next
tick.  Time to solution is measured from arrival to the result being on the
host.

A member's state in a batch is bit for bit the state it reaches alone with the
same tile shape, so a request's result does not depend on what else is being
served; across tile shapes it agrees to rounding.

The scheduling logic (``Server``) talks to an executor; ``PondExecutor``
drives the C ABI, and tests drive ``Server`` with a fake executor on the CPU.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import pond
from . import workloads as W


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    dim: int                # 1 or 2
    cfg: dict
    fields: tuple           # rho, ux, uy, T
    steps: int
    cells: int = 0
    admit_t: float | None = None
    finish_t: float | None = None
    status: str = "pending"  # pending, queued, running, done, rejected
    result: object = None
    flags: int = 0
    steps_done: int = 0      # steps advanced (all of them once done)

    def __post_init__(self):
        self.cells = int(self.cfg["nx"]) * int(self.cfg["ny"] if self.dim == 2 else 1)

    @property
    def latency(self):
        return None if self.finish_t is None else self.finish_t - self.arrival


class Server:
    """First-come first-served admission under a device-memory budget, one
    tick of at most ``tick_steps`` steps for every admitted request at a time."""

    def __init__(self, executor, budget_bytes: int, tick_steps: int = 64, clock=time.perf_counter,
                 sleep=time.sleep):
        if tick_steps < 1:
            raise ValueError("tick_steps must be >= 1")
        self.ex = executor
        self.budget = int(budget_bytes)
        self.tick_steps = int(tick_steps)
        self.clock = clock
        self.sleep = sleep
        self.peak_bytes = 0
        self.ticks = 0

    def run(self, requests, wall_limit: float | None = None):
        """Serves the requests until all are done, or until ``wall_limit``
        seconds after the start: then the requests still running are dropped
        from the device (status stays "running"), and those queued or not yet
        arrived keep "queued" / "pending"."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        pending = deque(reqs)
        queue = deque()
        active = []          # (request, handle, bytes)
        used = 0
        t0 = self.clock()
        self.stopped_at = None
        while pending or queue or active:
            now = self.clock() - t0
            if wall_limit is not None and now >= wall_limit:
                self.stopped_at = now
                for r, h, _ in active:
                    r.steps_done = r.steps - self.ex.remaining(h)
                    self.ex.abandon(h)
                break
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                r.status = "queued"
                queue.append(r)
            while queue:
                r = queue[0]
                need = self.ex.bytes_needed(r)
                if need > self.budget:
                    queue.popleft()
                    r.status = "rejected"
                    continue
                if used + need > self.budget or not self.ex.has_slot(r):
                    break
                queue.popleft()
                r.admit_t = self.clock() - t0
                r.status = "running"
                active.append((r, self.ex.admit(r), need))
                used += need
                self.peak_bytes = max(self.peak_bytes, used)
            if not active:
                if pending:
                    wait = pending[0].arrival - (self.clock() - t0)
                    if wait > 0:
                        self.sleep(wait)
                continue
            self.ex.tick([h for _, h, _ in active], self.tick_steps)
            self.ticks += 1
            still = []
            for r, h, need in active:
                if self.ex.remaining(h) == 0:
                    r.result, r.flags = self.ex.harvest(h)
                    r.finish_t = self.clock() - t0
                    r.status = "done"
                    r.steps_done = r.steps
                    used -= need
                else:
                    still.append((r, h, need))
            active = still
        return reqs


def summary(reqs, makespan: float | None = None):
    """p50/p99 time to solution (s) of the finished requests, aggregate MLUPS
    over the run (finished work over the makespan; with the steps advanced by
    requests still running when a wall-time limit stopped the run, in
    ``mlups_all_work``), counts by status."""
    done = [r for r in reqs if r.status == "done"]
    lat = np.array([r.latency for r in done]) if done else np.zeros(0)
    if makespan is None:
        makespan = max((r.finish_t for r in done), default=0.0) - min((r.arrival for r in reqs), default=0.0)
    work = sum(r.cells * r.steps for r in done)
    all_work = work + sum(r.cells * r.steps_done for r in reqs if r.status == "running")
    return {
        "requests": len(reqs), "done": len(done),
        "rejected": sum(1 for r in reqs if r.status == "rejected"),
        "running": sum(1 for r in reqs if r.status == "running"),
        "queued": sum(1 for r in reqs if r.status == "queued"),
        "not_arrived": sum(1 for r in reqs if r.status == "pending"),
        "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_s": float(lat.mean()) if len(lat) else None,
        "makespan_s": float(makespan),
        "mlups": work / makespan / 1e6 if makespan > 0 else None,
        "mlups_all_work": all_work / makespan / 1e6 if makespan > 0 else None,
        "cell_updates": int(work),
        "nonphysical": sum(1 for r in done if r.flags & pond.POND_FLAG_NONPHYSICAL),
    }


class PondExecutor:
    """Runs admitted requests as members of two pond batches (1D, 2D)."""

    @dataclass
    class Handle:
        req: Request
        sim: object
        dim: int
        remaining: int

    def __init__(self, precision: int = pond.POND_FP32_MIXED, capacity: int = 128,
                 graph_steps: int = 8, tile: int = 0, device=None):
        """tile 0: each batch's autotuner picks its 2D tile shape (results then
        agree with a solo run of the same request to rounding); a fixed tile
        equal to the solo default makes them agree bit for bit."""
        self.precision = precision
        self.capacity = capacity
        self.batches = {}
        for d in (1, 2):
            tune = pond.pond_tune_default()
            tune.graph_steps = graph_steps
            tune.tile = tile if d == 2 else 0  # a 1D batch has the one 252-cell tile
            self.batches[d] = pond.Batch(d, precision, capacity, tune, device=device)
        self.handles = {1: [], 2: []}   # in batch member order

    def _cfg(self, r):
        return dict(r.cfg, precision=self.precision)

    def bytes_needed(self, r):
        lat = pond.POND_D2Q16 if r.dim == 2 else pond.POND_D1Q4
        p = pond.params_from_config(self._cfg(r))
        return pond.pond_workspace_size(lat, (r.cfg["nx"], r.cfg["ny"] if r.dim == 2 else 1), p) + 256

    def has_slot(self, r):
        return len(self.handles[r.dim]) < self.capacity

    def admit(self, r):
        b = self.batches[r.dim]
        sim = pond.Sim(self._cfg(r), stream=b.stream)
        sim.init(*r.fields)
        b.add(sim)
        h = PondExecutor.Handle(r, sim, r.dim, int(r.steps))
        self.handles[r.dim].append(h)
        return h

    def tick(self, handles, tick_steps):
        with pond.nvtx_range("serve_tick"):
            self._tick(tick_steps)

    def _tick(self, tick_steps):
        for d in (1, 2):
            hs = self.handles[d]
            if not hs:
                continue
            steps = [min(h.remaining, tick_steps) for h in hs]
            self.batches[d].step(steps)   # asynchronous on the batch's stream
            for h, s in zip(hs, steps):
                h.remaining -= s

    def remaining(self, h):
        return h.remaining

    def harvest(self, h):
        m = h.sim.moments()                # waits for the batch stream
        flags = h.sim.flags()[1]
        self.batches[h.dim].remove(h.sim)
        self.handles[h.dim].remove(h)
        h.sim.close()
        return m, flags

    def abandon(self, h):
        """Drops a running request (the server's wall-time limit): it leaves
        its batch and its memory is freed, with no result."""
        self.batches[h.dim].remove(h.sim)
        self.handles[h.dim].remove(h)
        h.sim.close()

    def close(self):
        for b in self.batches.values():
            b.close()


def make_requests(n: int, rate: float, seed: int = 0, side_range_2d=(128, 1024),
                  n_range_1d=(256, 8192), steps_range=(500, 5000), frac_2d: float = 0.5):
    """Poisson arrivals at ``rate`` per second: Sod-type tubes (D1Q4, seeded
    left/right states) and 2D shock-bubble problems (D2Q16, seeded Mach number
    and bubble density ratio), each with a seeded number of steps."""
    g = W.rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += float(g.exponential(1.0 / rate))
        steps = int(g.integers(steps_range[0], steps_range[1] + 1))
        if g.random() < frac_2d:
            side = int(round(math.exp(g.uniform(math.log(side_range_2d[0]), math.log(side_range_2d[1])))))
            w = W.shock_bubble_2d(seed=int(g.integers(1 << 30)), n=side, steps=steps)
            dim = 2
        else:
            nx = int(round(math.exp(g.uniform(math.log(n_range_1d[0]), math.log(n_range_1d[1])))))
            w = W.random_tube_1d(seed=int(g.integers(1 << 30)), n=nx, steps=steps)
            dim = 1
        out.append(Request(i, t, dim, w["cfg"], (w["rho"], w["ux"], w["uy"], w["T"]), steps))
    return out
