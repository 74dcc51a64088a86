"""Multiscale f-lattice on the GPU (Sec. II.E lifting and projection, Sec.
IV.C switching): the same state and the same count of high-lattice cell
updates as the oracle, across tiles with ragged tails, boundaries (walls
included), limiters, the Grad projection, the quasi-equilibrium step and
Appendix C's flux form; the single-lattice limits;
the Lax tube of Sec. V.C.1; and the configurations it does not cover."""
import numpy as np
import pytest

import oracle
from paper_2302_00310_gb300 import pond
from paper_2302_00310_gb300 import workloads as W
from tests import riemann_exact as RE

pytestmark = pytest.mark.gpu
TOL = 1e-12
INFLOW = ((1.1, 0.5, -0.2, 0.8),) * 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pond.lib(build=True)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _gap_threshold(values, q=0.6, min_gap=1e-9):
    """A threshold near the q-quantile of the measures, in the middle of a
    gap between them, so that rounding cannot move a cell across it."""
    v = np.unique(np.asarray(values).ravel())
    i0 = int(q * (v.size - 1))
    lo, hi = max(i0 - v.size // 5, 0), min(i0 + v.size // 5, v.size - 2)
    gaps = v[lo + 1:hi + 2] - v[lo:hi + 1]
    i = lo + int(np.argmax(gaps))
    assert v[i + 1] - v[i] > min_gap * max(abs(v[i + 1]), 1e-300)
    return 0.5 * (v[i] + v[i + 1])


def _thresholds(cfg, fields, steps, min_gap=1e-9):
    """Thresholds clear of every cell's measures at the start of every step
    of the oracle run."""
    ocfg = oracle.Config.from_dict(dict(cfg, ms=1, ms_theta_u=-1.0, ms_theta_T=-1.0))
    st = oracle.init(ocfg, *fields)
    su_all, sT_all = [], []
    th = None
    for _ in range(2):  # the second pass follows the run with the chosen thresholds
        su_all, sT_all = [], []
        for _s in range(steps):
            su, sT = oracle.ms_measure(ocfg, st.ux, st.uy, st.T)
            su_all.append(su)
            sT_all.append(sT)
            st = oracle.run(ocfg, st, 1)
        th = (_gap_threshold(su_all, min_gap=min_gap), _gap_threshold(sT_all, min_gap=min_gap))
        ocfg = oracle.Config.from_dict(dict(cfg, ms=1, ms_theta_u=th[0], ms_theta_T=th[1]))
        st = oracle.init(ocfg, *fields)
    return th


WALLS_2D = ((0.0,) * 4, (0.0,) * 4, (0.0, 0.2, 0.0, 1.0), (0.0, -0.1, 0.0, 1.1))
WALLS_1D = ((0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.1), (0.0,) * 4, (0.0,) * 4)

MS_CASES = [
    # D, nx, ny, bc, limiter, grad_k, appc, mach, steps, other options
    (2, 37, 30, (0, 0, 0, 0), 0, 0, 0, 0.8, 3, {}),
    (2, 29, 33, (1, 1, 1, 1), 1, 1, 0, 1.0, 2, {}),
    (2, 24, 31, (2, 1, 0, 0), 0, 0, 1, 0.6, 2, {}),
    (2, 17, 45, (0, 0, 2, 2), 1, 1, 1, 0.9, 2, {}),
    (1, 300, 1, (1, 1, 0, 0), 0, 0, 0, 1.0, 3, {}),
    (1, 253, 1, (2, 1, 0, 0), 1, 0, 1, 0.8, 2, {}),
    # the quasi-equilibrium step (Pr != 1) and walls
    (2, 27, 31, (0, 0, 0, 0), 1, 1, 1, 0.8, 2, dict(prandtl=0.5)),
    (2, 30, 26, (1, 1, 3, 3), 0, 0, 0, 0.6, 2, dict(prandtl=0.71, inflow=WALLS_2D)),
    (2, 21, 35, (0, 0, 3, 3), 1, 1, 1, 0.6, 2, dict(inflow=WALLS_2D)),
    (1, 230, 1, (3, 3, 0, 0), 0, 0, 0, 0.5, 3, dict(prandtl=0.71, inflow=WALLS_1D)),
]


@pytest.mark.parametrize("case", range(len(MS_CASES)))
def test_multiscale_matches_oracle(case):
    D, nx, ny, bc, lim, gk, appc, mach, steps, extra = MS_CASES[case]
    walls = 3 in bc
    fields = W.random_state_grid(D, nx, ny, seed=150 + case, mach=mach, T=(0.7, 1.4) if walls else (0.5, 2.0))
    cfg = W._base(D, nx, ny, tau=5e-3, dx=1.0 / nx, limiter=lim, grad_k=gk, flux_appc=appc, bc=bc,
                  **dict(dict(inflow=INFLOW), **extra))
    cfg["dt"] = W.dt_from_cfl(fields[1], fields[2], fields[3], cfg["dx"], 0.4)
    thu, thT = _thresholds(cfg, fields, steps)
    cfg = dict(cfg, ms=1, ms_theta_u=thu, ms_theta_T=thT)
    ocfg = oracle.Config.from_dict(cfg)
    ost = oracle.run(ocfg, oracle.init(ocfg, *fields), steps)
    sim = pond.Sim(cfg)
    sim.init(*fields)
    sim.step(steps)
    f, g, ux, uy, T = sim.get_state()
    high = sim.ms_stats()
    flags = sim.flags()
    sim.close()
    cells = steps * nx * (ny if D == 2 else 1)
    assert 0.1 * cells < ost.report["ms_high"] < 0.9 * cells
    assert high == ost.report["ms_high"]
    errs = {"f": _rel(f, ost.f), "g": _rel(g, ost.g), "ux": _rel(ux, ost.ux), "T": _rel(T, ost.T)}
    if D == 2:
        errs["uy"] = _rel(uy, ost.uy)
    assert max(errs.values()) <= TOL, errs
    assert flags[1] & pond.POND_FLAG_NONPHYSICAL == 0


MIXED_CASES = [
    # D, nx, ny, bc, limiter, grad_k, steps, other options (default: Appendix C's flux form)
    (2, 37, 30, (0, 0, 0, 0), 0, 0, 3, {}),
    (2, 29, 33, (1, 1, 2, 1), 1, 1, 2, {}),
    (1, 300, 1, (1, 1, 0, 0), 0, 0, 3, {}),
    (2, 31, 27, (0, 0, 3, 3), 0, 0, 2, dict(prandtl=0.71, inflow=WALLS_2D)),
    # the main flux form: a low cell's energy flux in its own frame
    (2, 37, 30, (0, 0, 0, 0), 0, 0, 3, dict(flux_appc=0)),
    (2, 29, 33, (1, 1, 2, 1), 1, 1, 2, dict(flux_appc=0, prandtl=0.71)),
    (1, 300, 1, (1, 1, 0, 0), 0, 0, 3, dict(flux_appc=0)),
    (1, 120, 1, (3, 3, 0, 0), 1, 0, 3, dict(flux_appc=0, prandtl=0.71, inflow=WALLS_1D)),
    (2, 31, 27, (0, 0, 3, 3), 0, 0, 2, dict(flux_appc=0, prandtl=0.71, inflow=WALLS_2D)),
]


@pytest.mark.parametrize("case", range(len(MIXED_CASES)))
def test_multiscale_mixed_path(case):
    """The mixed path with the multiscale f-lattice, in Appendix C's form and
    in the main flux form (a low cell's energy flux taken in its own frame):
    the oracle's moments within the step bound 2e-6 and its count of
    high-lattice cell updates (thresholds clear of the measures by far more
    than FP32 rounding)."""
    D, nx, ny, bc, lim, gk, steps, extra = MIXED_CASES[case]
    walls = 3 in bc
    fields = W.random_state_grid(D, nx, ny, seed=190 + case, mach=0.8, T=(0.7, 1.4) if walls else (0.5, 2.0))
    cfg = W._base(D, nx, ny, tau=5e-3, dx=1.0 / nx, limiter=lim, grad_k=gk, bc=bc,
                  **dict(dict(inflow=INFLOW, flux_appc=1), **extra))
    cfg["dt"] = W.dt_from_cfl(fields[1], fields[2], fields[3], cfg["dx"], 0.4)
    thu, thT = _thresholds(cfg, fields, steps, min_gap=1e-4)
    cfg = dict(cfg, ms=1, ms_theta_u=thu, ms_theta_T=thT)
    ocfg = oracle.Config.from_dict(cfg)
    ost = oracle.run(ocfg, oracle.init(ocfg, *fields), steps)
    om = oracle.moments(ocfg, ost)
    sim = pond.Sim(dict(cfg, precision=pond.POND_FP32_MIXED))
    sim.init(*fields)
    sim.step(steps)
    gm = sim.moments()
    high = sim.ms_stats()
    sim.close()
    assert high == ost.report["ms_high"]
    for i in ((0, 1, 2, 3) if D == 2 else (0, 1, 3)):
        assert _rel(gm[i], om[i]) <= 2e-6, (i, _rel(gm[i], om[i]))


@pytest.mark.parametrize("D", [1, 2])
def test_single_lattice_limits(D):
    """All cells high: the plain D2Q16 kernel's state (to rounding: another
    instantiation); all cells low: the oracle's D2Q9 f-lattice step."""
    n = 40 if D == 2 else 300
    fields = W.random_state_grid(D, n, n, seed=7, mach=0.8)
    cfg = W._base(D, n, n, tau=5e-3, dx=1.0 / n, bc=(1, 1, 1, 1))
    cfg["dt"] = W.dt_from_cfl(fields[1], fields[2], fields[3], cfg["dx"], 0.3)
    out = {}
    for name, extra in (("plain", {}), ("high", dict(ms=1, ms_theta_u=-1.0, ms_theta_T=-1.0)),
                        ("low", dict(ms=1, ms_theta_u=1e30, ms_theta_T=1e30))):
        sim = pond.Sim(dict(cfg, **extra))
        sim.init(*fields)
        sim.step(3)
        out[name] = (sim.get_state(), sim.moments(), sim.ms_stats())
        sim.close()
    cells = 3 * n * (n if D == 2 else 1)
    assert out["high"][2] == cells and out["low"][2] == 0
    for a, b in zip(out["high"][0], out["plain"][0]):
        assert _rel(a, b) <= 1e-13
    o3 = oracle.Config.from_dict(dict(cfg, qf=3))
    ost = oracle.run(o3, oracle.init(o3, *fields), 3)
    om = oracle.moments(o3, ost)
    for k in ((0, 1, 2, 3) if D == 2 else (0, 1, 3)):
        assert _rel(out["low"][1][k], om[k]) <= TOL, k


def test_lax_tube_on_the_gpu():
    """Sec. V.C.1 at L = 400: the multiscale run's density error against the
    exact solution equals the oracle's, as does its share of high-lattice
    cell updates (to the cells whose measure rounding could move across the
    threshold over 2,000 steps)."""
    left, right = (0.445, 0.698, 3.528), (0.5, 0.0, 0.571)
    w = W.lax_1d(n=400)
    cfg = dict(w["cfg"], ms=1, ms_theta_u=0.05, ms_theta_T=0.05)
    exact = RE.solution(left, right, w["x"], w["t_end"])[0]
    ocfg = oracle.Config.from_dict(cfg)
    ost = oracle.run(ocfg, oracle.init(ocfg, w["rho"], w["ux"], w["uy"], w["T"]), w["steps"])
    oerr = float(np.mean(np.abs(oracle.moments(ocfg, ost)[0][0] - exact)))
    sim = pond.Sim(cfg)
    sim.init(w["rho"], w["ux"], w["uy"], w["T"])
    sim.step(w["steps"])
    rho = np.asarray(sim.moments()[0]).ravel()
    high = sim.ms_stats()
    sim.close()
    gerr = float(np.mean(np.abs(rho - exact)))
    assert abs(gerr - oerr) <= 1e-3 * oerr
    assert abs(high - ost.report["ms_high"]) <= 1e-3 * ost.report["ms_high"]


@pytest.mark.parametrize("bad", [dict(iterative=1), dict(tile=6), dict(qf=5)])
def test_multiscale_rejects_what_it_does_not_cover(bad):
    fields = W.random_state_grid(2, 16, 16, seed=1)
    cfg = W._base(2, 16, 16, tau=5e-3, dx=1.0 / 16, inflow=((0.0, 0.1, 0.0, 1.0),) * 4)
    cfg["dt"] = 1e-4
    cfg = dict(cfg, ms=1, ms_theta_u=0.1, ms_theta_T=0.1, **bad)
    with pytest.raises(pond.PondError):
        sim = pond.Sim(cfg)
        sim.init(*fields)
        sim.close()


def test_multiscale_context_is_not_batched():
    fields = W.random_state_grid(2, 16, 16, seed=2)
    cfg = W._base(2, 16, 16, tau=5e-3, dx=1.0 / 16)
    cfg["dt"] = 1e-4
    b = pond.Batch(2, pond.POND_FP64, 4)
    sim = pond.Sim(dict(cfg, ms=1, ms_theta_u=0.1, ms_theta_T=0.1), stream=b.stream)
    sim.init(*fields)
    with pytest.raises(pond.PondError):
        b.add(sim)
    b.close()
    sim.close()


def test_reported_tile_is_the_shape_that_runs():
    """pond_info's tile code names the kernel shape a context steps with.  On
    a 512^2 grid (2,368 tiles of 8x14, at least four waves of three CTAs per
    SM on a 152-SM GPU) a plain mixed context takes the capped tile 11, the
    FP64 one tile 10, and the multiscale and g-on-f contexts, whose kernels
    have the one 8x14 two-CTA shape, report that shape's code 10."""
    import torch

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 512
    tiles = (n // 8) * ((n + 13) // 14)
    cfg = W._base(2, n, n, tau=1e-3, dt=1e-4, bc=(0, 0, 0, 0))
    mixed = dict(cfg, precision=pond.POND_FP32_MIXED)
    expect = [(dict(cfg), 10), (mixed, 11 if tiles >= 12 * sms else 10),
              (dict(mixed, ms=1, ms_theta_u=0.05, ms_theta_T=0.05), 10), (dict(mixed, qg=4), 10),
              (dict(cfg, ms=1, ms_theta_u=0.05, ms_theta_T=0.05), 10)]
    for c, code in expect:
        sim = pond.Sim(c)
        try:
            assert sim.info()[2] == code, c
        finally:
            sim.close()
