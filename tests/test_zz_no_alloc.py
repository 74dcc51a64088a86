"""pond_step_noalloc(): the step for callers that may not call cudaMalloc
(graph capture in global mode, pool-owned device memory, latency-critical
loops).  It must give the same state as the context entry point pond_step(),
on two calls in a row, using only its static device scratch.

Collected last on purpose (file name), so that a run stopping at the first
failure has run every other test first; it also passes alone in a fresh
process."""
import numpy as np
import pytest

from paper_2302_00310_gb300 import pond
from paper_2302_00310_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    pond.lib(build=True)
    return t


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _device_state(torch, sim):
    shp = (sim.ny, sim.nx)
    dev = [torch.empty((sim.Qf,) + shp, dtype=torch.float64, device="cuda"),
           torch.empty((sim.Qg,) + shp, dtype=torch.float64, device="cuda")]
    dev += [torch.empty(shp, dtype=torch.float64, device="cuda") for _ in range(3)]
    pond.pond_get_state(sim.ctx, dev[0], dev[1], dev[2], dev[3] if sim.D == 2 else None, dev[4])
    return dev


def _walled_ragged_2d():
    """A 90 x 77 channel: walls on the y sides (the lower one moving), zero
    gradient on the x sides; neither side a multiple of the 8x8 tile."""
    nx, ny = 90, 77
    rho, ux, uy, T = W.random_state_grid(2, nx, ny, seed=91, mach=0.6, T=(0.8, 1.3))
    walls = ((0.0,) * 4, (0.0,) * 4, (0.0, 0.25, 0.0, 0.95), (0.0, 0.0, 0.0, 1.1))
    cfg = W._base(2, nx, ny, tau=5e-3, dx=1.0 / nx, prandtl=0.71, bc=(1, 1, 3, 3), inflow=walls)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4)
    return {"cfg": cfg, "rho": rho, "ux": ux, "uy": uy, "T": T}


@pytest.mark.parametrize("case", ["pulse2d", "walls2d", "sod1d"])
def test_noalloc_matches_context_step_on_two_calls(torch, case):
    if case == "pulse2d":
        w = W.pulse_2d(n=96, seed=3)
        w["cfg"]["prandtl"], w["cfg"]["tau"] = 0.71, 2e-3
    elif case == "walls2d":
        w = _walled_ragged_2d()
    else:
        w = W.sod_1d(n=1000, cfl=0.4)
    D = 1 if case == "sod1d" else 2
    cfg = w["cfg"]
    sim = pond.Sim(cfg)
    sim.init(w["rho"], w["ux"], w["uy"], w["T"])
    state = _device_state(torch, sim)  # the caller's state, on the device
    sim.step(3)
    ref1 = sim.get_state()
    sim.step(4)
    ref2 = sim.get_state()
    sim.close()

    params = pond.params_from_config(cfg)
    lat = pond.POND_D2Q16 if D == 2 else pond.POND_D1Q4
    dims = (cfg["nx"], cfg["ny"] if D == 2 else 1)
    stream = torch.cuda.Stream()
    uy = state[3] if D == 2 else None
    for nsteps, ref in ((3, ref1), (4, ref2)):
        st, flags = pond.pond_step_noalloc(lat, dims, params, state[0], state[1], state[2], uy,
                                           state[4], nsteps, stream=stream.cuda_stream)
        assert st == pond.POND_OK and flags & pond.POND_FLAG_NONPHYSICAL == 0
        got = [t.cpu().numpy() for t in state]
        for k, (a, b) in enumerate(zip(got, ref)):
            if D == 1 and k == 3:
                continue
            assert _rel(a, b) <= TOL, (nsteps, k, _rel(a, b))


def test_noalloc_rejects_a_state_larger_than_its_scratch(torch):
    p = pond.pond_params_default()
    p.dt = 1e-4
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(pond.PondError) as e:
        pond.pond_step_noalloc(pond.POND_D2Q16, (512, 512), p, dummy, dummy, dummy, dummy, dummy, 1)
    assert e.value.status == pond.POND_E_NOMEM
    p.precision = pond.POND_FP32_MIXED
    with pytest.raises(pond.PondError) as e:
        pond.pond_step_noalloc(pond.POND_D2Q16, (16, 16), p, dummy, dummy, dummy, dummy, dummy, 1)
    assert e.value.status == pond.POND_E_INVAL


def test_noalloc_refuses_flags_while_its_stream_is_captured(torch):
    """Reading the flags synchronises the stream, which a capture forbids: the
    call returns POND_E_INVAL before any work, and the capture stays valid."""
    w = W.sod_1d(n=64, cfl=0.4)
    sim = pond.Sim(w["cfg"])
    sim.init(w["rho"], w["ux"], w["uy"], w["T"])
    state = _device_state(torch, sim)
    sim.close()
    params = pond.params_from_config(w["cfg"])
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    marker = torch.zeros(1, device="cuda")
    status = None
    with torch.cuda.graph(graph, stream=stream):
        marker += 1.0
        try:
            pond.pond_step_noalloc(pond.POND_D1Q4, (64, 1), params, state[0], state[1], state[2],
                                   None, state[4], 1, stream=stream.cuda_stream, want_flags=True)
        except pond.PondError as e:
            status = e.status
    assert status == pond.POND_E_INVAL
    graph.replay()
    torch.cuda.synchronize()
    assert float(marker.item()) == 1.0  # the one captured increment, replayed once
