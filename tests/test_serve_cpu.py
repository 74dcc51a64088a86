"""Host logic of the continuous-batching server, driven by a fake executor
and a fake clock on the CPU (no GPU)."""
import numpy as np
import pytest

from paper_2302_00310_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeExecutor:
    """Each tick costs 1 ms per million cell updates it performs."""

    def __init__(self, clock, slots=100):
        self.clock = clock
        self.slots = slots
        self.active = {}
        self.log = []

    def bytes_needed(self, r):
        return r.cells * 100

    def has_slot(self, r):
        return len(self.active) < self.slots

    def admit(self, r):
        self.active[r.rid] = [r, r.steps]
        self.log.append(("admit", r.rid, self.clock.t))
        return r.rid

    def tick(self, handles, tick_steps):
        work = 0
        for h in handles:
            s = min(self.active[h][1], tick_steps)
            self.active[h][1] -= s
            work += s * self.active[h][0].cells
        self.clock.t += 1e-3 * work / 1e6 + 1e-5

    def remaining(self, h):
        return self.active[h][1]

    def harvest(self, h):
        r, _ = self.active.pop(h)
        self.log.append(("done", r.rid, self.clock.t))
        return ("moments", r.rid), 0

    def abandon(self, h):
        r, _ = self.active.pop(h)
        self.log.append(("abandon", r.rid, self.clock.t))


def _req(rid, t, nx, steps, dim=2):
    cfg = {"nx": nx, "ny": nx if dim == 2 else 1}
    return serve.Request(rid, t, dim, cfg, (), steps)


def test_every_request_finishes_with_its_latency():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    reqs = [_req(i, 0.01 * i, 64 + 8 * i, 100 + 10 * i) for i in range(20)]
    out = serve.Server(ex, budget_bytes=10**9, tick_steps=32, clock=clk, sleep=clk.sleep).run(reqs)
    assert all(r.status == "done" for r in out)
    for r in out:
        assert r.admit_t >= r.arrival and r.finish_t > r.admit_t
        assert r.result == ("moments", r.rid)
    s = serve.summary(out)
    lat = sorted(r.latency for r in out)
    assert s["done"] == 20 and s["p50_s"] == pytest.approx(np.percentile(lat, 50))
    assert s["cell_updates"] == sum(r.cells * r.steps for r in out)


def test_admission_respects_the_memory_budget_in_arrival_order():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    reqs = [_req(i, 0.0, 100, 200) for i in range(6)]       # 1e6 bytes each
    srv = serve.Server(ex, budget_bytes=2_500_000, tick_steps=50, clock=clk, sleep=clk.sleep)
    out = srv.run(reqs)
    assert srv.peak_bytes <= 2_500_000
    admits = [rid for kind, rid, _ in ex.log if kind == "admit"]
    assert admits == sorted(admits)                         # first come, first served
    # never more than two resident at once
    live, peak = 0, 0
    for kind, _, _ in ex.log:
        live += 1 if kind == "admit" else -1
        peak = max(peak, live)
    assert peak == 2 and all(r.status == "done" for r in out)


def test_request_larger_than_the_budget_is_rejected_not_blocking():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    reqs = [_req(0, 0.0, 1000, 10), _req(1, 0.0, 10, 10)]
    out = serve.Server(ex, budget_bytes=50_000, clock=clk, sleep=clk.sleep).run(reqs)
    assert out[0].status == "rejected" and out[1].status == "done"
    assert serve.summary(out)["rejected"] == 1


def test_late_arrivals_join_a_running_batch():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    reqs = [_req(0, 0.0, 512, 4000), _req(1, 0.05, 32, 100)]
    out = serve.Server(ex, budget_bytes=10**9, tick_steps=64, clock=clk, sleep=clk.sleep).run(reqs)
    a0 = [t for k, rid, t in ex.log if k == "admit" and rid == 1][0]
    d0 = [t for k, rid, t in ex.log if k == "done" and rid == 0][0]
    # the short request was admitted and finished while the long one ran
    assert a0 < d0 and out[1].finish_t < out[0].finish_t


def test_idle_server_waits_for_the_next_arrival():
    clk = FakeClock()
    ex = FakeExecutor(clk)
    reqs = [_req(0, 5.0, 16, 10)]
    out = serve.Server(ex, budget_bytes=10**9, clock=clk, sleep=clk.sleep).run(reqs)
    assert out[0].admit_t >= 5.0 and out[0].status == "done"


def test_request_stream_is_seeded_and_poisson():
    a = serve.make_requests(40, rate=200.0, seed=3, side_range_2d=(16, 32), n_range_1d=(64, 128),
                            steps_range=(5, 10))
    b = serve.make_requests(40, rate=200.0, seed=3, side_range_2d=(16, 32), n_range_1d=(64, 128),
                            steps_range=(5, 10))
    assert [(r.arrival, r.dim, r.cells, r.steps) for r in a] == [(r.arrival, r.dim, r.cells, r.steps) for r in b]
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert np.all(gaps > 0) and 0.002 < gaps.mean() < 0.01
    assert {r.dim for r in a} == {1, 2}
    for r in a:
        assert 5 <= r.steps <= 10
        n = r.cfg["nx"]
        assert (16 <= n <= 32) if r.dim == 2 else (64 <= n <= 128)


def test_nvtx_ranges_nest_and_never_raise_on_the_host():
    """The NVTX ranges around enqueued steps and serve ticks are markers only:
    on a host without a GPU they neither raise nor leave a range open."""
    from paper_2302_00310_gb300 import pond

    with pond.nvtx_range("outer"):
        with pond.nvtx_range("inner"):
            pass
    with pytest.raises(ValueError):
        with pond.nvtx_range("raising"):
            raise ValueError("propagates")


def test_wall_limit_stops_and_reports_the_queue():
    """An offered load beyond the executor's rate, served for a fixed wall
    time: requests finished by then are done, the running ones are dropped
    from the device, the rest stay queued or not yet arrived."""
    clock = FakeClock()
    ex = FakeExecutor(clock, slots=2)
    srv = serve.Server(ex, budget_bytes=10**12, tick_steps=100, clock=clock, sleep=clock.sleep)
    # each request: 1e6 cell updates per 100-step tick -> 1 ms per tick, 10 ticks
    reqs = [_req(i, 0.001 * i, 100, 1000) for i in range(40)]
    out = srv.run(reqs, wall_limit=0.05)
    s = serve.summary(out, makespan=srv.stopped_at)
    assert srv.stopped_at is not None and srv.stopped_at >= 0.05
    assert 0 < s["done"] < 40 and s["running"] == 2
    assert s["done"] + s["running"] + s["queued"] + s["not_arrived"] == 40
    assert not ex.active  # nothing left on the device
    assert sum(1 for e in ex.log if e[0] == "abandon") == 2
    # the running requests' steps count in mlups_all_work, not in mlups
    running = [r for r in out if r.status == "running"]
    assert all(0 < r.steps_done < r.steps for r in running)
    partial = sum(r.cells * r.steps_done for r in running)
    assert abs(s["mlups_all_work"] - s["mlups"] - partial / s["makespan_s"] / 1e6) < 1e-9 * s["mlups_all_work"]
