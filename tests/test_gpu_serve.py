"""The continuous-batching server on the GPU: every request's result is bit
for bit the result of running it alone, whatever else was being served."""
import numpy as np
import pytest

from paper_2302_00310_gb300 import pond, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    pond.lib(build=True)
    return t


def _solo_tile(precision):
    return 10  # pond_params.tile default in 2D for grids of these sizes


@pytest.mark.parametrize("precision,autotune", [(pond.POND_FP32_MIXED, False), (pond.POND_FP64, False),
                                                (pond.POND_FP32_MIXED, True)])
def test_each_result_is_the_same_alone_and_in_the_mix(torch, precision, autotune):
    """With the solo tile shape a served result equals the request run alone
    bit for bit; with the autotuner free to pick another shape, to the stated
    FP32 step bound."""
    reqs = serve.make_requests(10, rate=400.0, seed=5, side_range_2d=(24, 72),
                               n_range_1d=(64, 400), steps_range=(20, 90))
    ex = serve.PondExecutor(precision=precision, capacity=6, graph_steps=4,
                            tile=0 if autotune else _solo_tile(precision))
    srv = serve.Server(ex, budget_bytes=64 << 20, tick_steps=16)
    out = srv.run(reqs)
    ex.close()
    s = serve.summary(out)
    assert s["done"] == 10 and s["p99_s"] >= s["p50_s"] > 0
    for r in out:
        sim = pond.Sim(dict(r.cfg, precision=precision))
        sim.init(*r.fields)
        sim.step(r.steps)
        alone = sim.moments()
        sim.close()
        # velocity components are measured against the flow's velocity scale
        # (the larger component's maximum): a component that is nearly zero
        # everywhere carries rounding of the size of the other one's
        vscale = max(np.max(np.abs(alone[1])), np.max(np.abs(alone[2])) if r.dim == 2 else 0.0)
        for i, (a, b) in enumerate(zip(r.result, alone)):
            if r.dim == 1 and i == 2:
                continue
            if autotune:
                scale = vscale if i in (1, 2) else np.max(np.abs(b))
                assert np.max(np.abs(a - b)) <= 2e-6 * max(scale, 1e-30), (r.rid, i)
            else:
                assert np.array_equal(a, b), r.rid


def test_budget_limits_residency_on_the_device(torch):
    reqs = serve.make_requests(6, rate=1000.0, seed=8, side_range_2d=(64, 64),
                               n_range_1d=(256, 256), steps_range=(16, 16), frac_2d=1.0)
    ex = serve.PondExecutor(capacity=8, graph_steps=4)
    one = ex.bytes_needed(reqs[0])
    srv = serve.Server(ex, budget_bytes=2 * one + 1, tick_steps=8)
    out = srv.run(reqs)
    ex.close()
    assert srv.peak_bytes <= 2 * one + 1
    assert all(r.status == "done" for r in out)
    admits = sorted(out, key=lambda r: r.admit_t)
    assert [r.rid for r in admits] == sorted(r.rid for r in out)
