"""GPU parity: the CUDA path against the FP64 oracle, element by element, on
the same seeded inputs (both sides initialise from the same primitive
fields).  FP64 path tolerance: max|x_gpu - x_oracle| / max|x_oracle| <= 1e-12
per field (populations, frame)."""
import math

import numpy as np
import pytest

import oracle
from paper_2302_00310_gb300 import pond
from paper_2302_00310_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pond.lib(build=True)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _run_both(cfg, rho, ux, uy, T, steps, tile=0):
    ocfg = oracle.Config.from_dict(cfg)
    ost = oracle.run(ocfg, oracle.init(ocfg, rho, ux, uy, T), steps)
    c = dict(cfg, tile=tile)
    sim = pond.Sim(c)
    sim.init(rho, ux, uy, T)
    sim.step(steps)
    got = sim.get_state()
    flags = sim.flags() + sim.iter_stats()  # (status, flags, max cfl, noconv, evals, traces, max)
    sim.close()
    return ost, got, flags


def _compare(ost, got, D, tol=TOL):
    f, g, ux, uy, T = got
    errs = {"f": _rel(f, ost.f), "g": _rel(g, ost.g), "ux": _rel(ux, ost.ux), "T": _rel(T, ost.T)}
    if D == 2:
        errs["uy"] = _rel(uy, ost.uy)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, errs
    return errs


CASES_1D = [
    # nx, bc, prandtl, limiter, appc, mach, steps
    (300, (1, 1, 1, 1), 1.0, 0, 0, 0.8, 1),
    (300, (0, 0, 0, 0), 0.71, 1, 0, 1.0, 3),
    (253, (2, 1, 1, 1), 1.0, 0, 1, 0.5, 2),
    (2, (1, 1, 1, 1), 1.0, 0, 0, 0.5, 2),
    (505, (0, 0, 0, 0), 0.5, 0, 1, 1.0, 5),
]


@pytest.mark.parametrize("case", range(len(CASES_1D)))
def test_1d_random_state_matches_oracle(case):
    nx, bc, pr, lim, appc, mach, steps = CASES_1D[case]
    rho, ux, uy, T = W.random_state_grid(1, nx, 1, seed=10 + case, mach=mach)
    cfg = W._base(1, nx, 1, tau=5e-3, dx=1.0 / nx, prandtl=pr, limiter=lim, flux_appc=appc, bc=bc,
                  inflow=((1.2, 0.4, 0.0, 0.9),) * 4)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4)
    ost, got, flags = _run_both(cfg, rho, ux, uy, T, steps)
    _compare(ost, got, 1)
    assert flags[1] & pond.POND_FLAG_NONPHYSICAL == 0


CASES_2D = [
    # nx, ny, bc, prandtl, limiter, grad_k, appc, mach, steps, tile
    (37, 29, (0, 0, 0, 0), 1.0, 0, 0, 0, 0.8, 1, 2),
    (37, 29, (1, 1, 1, 1), 0.71, 1, 0, 0, 1.2, 2, 3),
    (21, 40, (2, 1, 1, 1), 1.0, 0, 1, 0, 0.6, 2, 4),
    (18, 17, (0, 0, 1, 1), 0.71, 0, 0, 1, 1.0, 3, 2),
    (2, 2, (0, 0, 0, 0), 1.0, 0, 0, 0, 0.5, 2, 2),
    (33, 35, (1, 2, 2, 1), 0.5, 1, 1, 1, 0.9, 2, 3),
    (27, 41, (0, 0, 1, 1), 0.71, 1, 0, 0, 1.0, 2, 5),
    (19, 37, (1, 1, 0, 0), 1.0, 0, 1, 1, 1.0, 2, 6),
    (29, 35, (2, 1, 0, 0), 0.71, 0, 0, 0, 1.0, 2, 9),
]


@pytest.mark.parametrize("case", range(len(CASES_2D)))
def test_2d_random_state_matches_oracle(case):
    nx, ny, bc, pr, lim, gk, appc, mach, steps, tile = CASES_2D[case]
    rho, ux, uy, T = W.random_state_grid(2, nx, ny, seed=20 + case, mach=mach)
    cfg = W._base(2, nx, ny, tau=5e-3, dx=1.0 / nx, prandtl=pr, limiter=lim, grad_k=gk,
                  flux_appc=appc, bc=bc, inflow=((1.1, 0.5, -0.2, 0.8),) * 4)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4)
    ost, got, flags = _run_both(cfg, rho, ux, uy, T, steps, tile=tile)
    _compare(ost, got, 2)


AT_REST_CASES = [
    # D, nx, ny, qf, limiter, iterative, steps, tile
    (2, 37, 29, 4, 0, 0, 3, 2),
    (2, 33, 35, 4, 1, 0, 2, 6),
    (2, 21, 19, 5, 0, 0, 2, 0),
    (2, 25, 23, 4, 0, 1, 2, 0),
    (1, 300, 1, 4, 1, 0, 3, 0),
]
AT_REST_MODES = ("xband", "yband", "rest", "all")


def at_rest_state(D, nx, ny, seed, mode):
    """Random fields with a band of cells at u_x = 0 ("xband"), (2D) a band
    at u_y = 0 ("yband"), a uniform gas at rest (rho = T = 1) in one quarter
    (half in 1D: "rest"), or all three ("all"): many faces have u_F,n = 0
    exactly, so the zero node of the D2Q9 / D1Q3 g-lattice (and of D2Q25's
    f-lattice) sits at v_n = 0 there."""
    rho, ux, uy, T = W.random_state_grid(D, nx, ny, seed=seed, mach=0.8, T=(0.7, 1.4))
    if mode in ("xband", "all"):
        ux[:, nx // 4: nx // 2] = 0.0
    if D == 2 and mode in ("yband", "all"):
        uy[ny // 2:, :] = 0.0
    if mode in ("rest", "all"):
        if D == 2:
            for a in (rho, T):
                a[ny // 2:, nx // 2:] = 1.0
            ux[ny // 2:, nx // 2:], uy[ny // 2:, nx // 2:] = 0.0, 0.0
        else:
            rho[:, nx // 2:], T[:, nx // 2:], ux[:, nx // 2:] = 1.0, 1.0, 0.0
    return rho, ux, uy, T


@pytest.mark.parametrize("mode", AT_REST_MODES)
@pytest.mark.parametrize("case", range(len(AT_REST_CASES)))
@pytest.mark.parametrize("precision", [pond.POND_FP64, pond.POND_FP32_MIXED])
def test_faces_at_rest_match_oracle(case, precision, mode):
    """The zero node at v_n = 0 takes the mean of its two one-sided traces
    (in line; the other nodes keep their upwind trace): the FP64 path gives
    the oracle's state to 1e-12, the mixed path its moments within 2e-6.

    The combined state runs one step only.  The choice of the upwind side
    jumps at v_n = 0, so both sides must see the same exact zeros: the
    kernel keeps a uniform gas at rest at u = 0 exactly (its momentum is a
    Hermite coefficient), while the oracle, summing populations, leaves
    rounding noise of ~1e-17 in it after a step.  Beside the cells of the
    x-band that are at rest in both components, with other densities and
    temperatures, that noise picks one side where the kernel takes the mean:
    a first-order difference, 1e-4 after the second step.  Alone, each
    feature keeps the same exact zeros on both sides for several steps.  The
    iterated frame (case 3) stops where successive frames differ by less than
    iter_tol = 1e-10, so its last iterate differs by up to ~1e-11 (FP64); on
    the mixed path a face whose zero node sits near v_n = 0 can change its
    upwind side between iterates, so the bound of the iterated frame's
    cycling faces, 1e-3, applies (measured 7.1e-5)."""
    D, nx, ny, qf, lim, it, steps, tile = AT_REST_CASES[case]
    if D == 1 and mode == "yband":
        pytest.skip("no y-axis in 1D")
    if mode == "all":
        steps = 1
    rho, ux, uy, T = at_rest_state(D, nx, ny, 150 + case, mode)
    cfg = W._base(D, nx, ny, qf=qf, tau=5e-3, dx=1.0 / nx, prandtl=0.71, limiter=lim, bc=(1, 1, 1, 1),
                  iterative=it, iter_tol=1e-10, iter_max=12)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4, c_max=W.C_MAX_D1Q5 if qf == 5 else W.C_MAX_D1Q4)
    if precision == pond.POND_FP64:
        ost, got, flags = _run_both(cfg, rho, ux, uy, T, steps, tile=tile)
        _compare(ost, got, D, tol=1e-10 if it else TOL)
    else:
        oc = oracle.Config.from_dict(cfg)
        om = oracle.moments(oc, oracle.run(oc, oracle.init(oc, rho, ux, uy, T), steps))
        sim = pond.Sim(dict(cfg, precision=precision, tile=tile))
        sim.init(rho, ux, uy, T)
        sim.step(steps)
        gm, flags = sim.moments(), sim.flags()
        sim.close()
        errs = [_rel(gm[i], om[i]) for i in ((0, 1, 2, 3) if D == 2 else (0, 1, 3))]
        print("MEASURED at_rest_case%d_%s_mixed linf %.3e" % (case, mode, max(errs)))
        assert max(errs) <= (1e-3 if it else 2e-6), errs
    assert flags[1] & pond.POND_FLAG_NONPHYSICAL == 0


@pytest.mark.parametrize("D,mach,gk", [(1, 2.0, 0), (2, 1.5, 1)])
def test_violent_state_is_flagged_like_the_oracle(D, mach, gk):
    """Random per-cell velocities at Mach 1.5-2 drive an interface temperature
    negative: both sides report the state as nonphysical."""
    n = 505 if D == 1 else 33
    rho, ux, uy, T = W.random_state_grid(D, n, n if D == 2 else 1, seed=14 if D == 1 else 25, mach=mach)
    cfg = W._base(D, n, n, tau=5e-3, dx=1.0 / n, prandtl=0.5, grad_k=gk, flux_appc=1,
                  bc=(0, 0, 0, 0) if D == 1 else (1, 2, 2, 1), inflow=((1.1, 0.5, -0.2, 0.8),) * 4)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4)
    ost, got, flags = _run_both(cfg, rho, ux, uy, T, 2)
    assert ost.report["flags"] & oracle.FLAG_NONPHYSICAL
    assert flags[0] == pond.POND_E_NONPHYSICAL and flags[1] & pond.POND_FLAG_NONPHYSICAL


def test_sod_full_run_matches_oracle():
    """The 400-cell Sod tube, 250 steps to t = 0.2 (config time step)."""
    w = W.sod_1d()
    ost, got, flags = _run_both(w["cfg"], w["rho"], w["ux"], w["uy"], w["T"], w["steps"])
    _compare(ost, got, 1)
    # the same CFL bookkeeping as the oracle
    assert abs(flags[2] - ost.report["max_cfl"]) < 1e-12 * ost.report["max_cfl"]
    assert flags[1] & pond.POND_FLAG_CFL  # CFL ~ 1.09 > 1 at the config time step


def test_config3_few_steps_matches_oracle():
    w = W.config3_2d(n=40, prandtl=0.71)
    w["cfg"]["tau"] = 2e-3
    ost, got, _ = _run_both(w["cfg"], w["rho"], w["ux"], w["uy"], w["T"], 5)
    _compare(ost, got, 2)


def _window_oracle(cfg, fields, j, k, steps):
    """Oracle run on the (4 steps + 1)^2 window around cell (j, k) of a periodic
    grid; the centre cell depends only on cells within 2 per step."""
    r = 2 * steps
    ny, nx = fields[0].shape
    jj = (np.arange(j - r, j + r + 1)) % nx
    kk = (np.arange(k - r, k + r + 1)) % ny
    sub = [np.ascontiguousarray(a[np.ix_(kk, jj)]) for a in fields]
    c = dict(cfg, nx=2 * r + 1, ny=2 * r + 1, bc=(1, 1, 1, 1))
    ocfg = oracle.Config.from_dict(c)
    st = oracle.run(ocfg, oracle.init(ocfg, *sub), steps)
    return st.f[:, r, r], st.g[:, r, r], st.ux[r, r], st.uy[r, r], st.T[r, r]


@pytest.mark.parametrize("steps", [1, 2])
def test_pulse_full_size_sampled_cells_match_oracle(steps):
    """256^2 periodic pulse in the benchmark's launch configuration; 24 seeded
    cells checked against the oracle one by one."""
    w = W.pulse_2d(n=256, seed=0)
    sim = pond.Sim(w["cfg"])
    sim.init(w["rho"], w["ux"], w["uy"], w["T"])
    sim.step(steps)
    f, g, ux, uy, T = sim.get_state()
    sim.close()
    rng = np.random.default_rng(5)
    fields = (w["rho"], w["ux"], w["uy"], w["T"])
    for j, k in rng.integers(0, 256, (24, 2)):
        of, og, oux, ouy, oT = _window_oracle(w["cfg"], fields, int(j), int(k), steps)
        assert _rel(f[:, k, j], of) <= TOL
        assert _rel(g[:, k, j], og) <= TOL
        assert abs(ux[k, j] - oux) <= TOL * abs(oux) and abs(T[k, j] - oT) <= TOL * oT


def test_pulse_full_run_conserves_and_advects():
    """1000 steps of the 256^2 pulse: totals conserved to rounding (Appendix C)
    and the density profile translated with the flow (Euler entropy wave)."""
    w = W.pulse_2d(n=256, seed=0, steps=1000)
    sim = pond.Sim(w["cfg"])
    sim.init(w["rho"], w["ux"], w["uy"], w["T"])
    r0, x0, y0, t0 = sim.moments()
    sim.step(w["steps"])
    r1, x1, y1, t1 = sim.moments()
    st, flags, cfl, _ = sim.flags()
    dt = sim.info()[0]
    sim.close()
    assert st == pond.POND_OK and not flags & pond.POND_FLAG_NONPHYSICAL
    cv = 1 / 0.4
    tot = lambda r, u, v, t: np.array([r.sum(), (r * u).sum(), (r * v).sum(),
                                       (cv * r * t + 0.5 * r * (u * u + v * v)).sum()])
    a, b = tot(r0, x0, y0, t0), tot(r1, x1, y1, t1)
    assert np.max(np.abs(a - b) / np.abs(a)) < 1e-11
    # exact solution: initial profile moved by u t (periodic)
    n = 256
    t_end = dt * w["steps"]
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    prof = np.zeros((n, n))
    U, V = w["velocity"]
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            dxp = (X - U * t_end - w["centre"][0]) % 1.0 - sx
            dyp = (Y - V * t_end - w["centre"][1]) % 1.0 - sy
            prof += np.exp(-(dxp**2 + dyp**2) / (2 * w["sigma"] ** 2))
    exact = 1 + 0.1 * prof
    l1 = np.mean(np.abs(r1 - exact)) / np.mean(exact - 1)
    assert l1 < 0.05, l1


def test_uniform_flow_stays_uniform_on_gpu():
    n = 20
    cs = math.sqrt(1.4 * 0.7)
    shp = (n, n)
    rho, T = np.full(shp, 1.3), np.full(shp, 0.7)
    ux, uy = np.full(shp, 5 * cs * 0.8), np.full(shp, 5 * cs * 0.6)
    cfg = W._base(2, n, n, tau=1e-3, dx=1.0 / n, bc=(0, 0, 0, 0))
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.5)
    sim = pond.Sim(cfg)
    sim.init(rho, ux, uy, T)
    sim.step(10)
    r, a, b, t = sim.moments()
    sim.close()
    assert np.max(np.abs(r - 1.3)) < 1e-13 and np.max(np.abs(t - 0.7)) < 1e-13
    assert np.max(np.abs(a - ux)) < 1e-12


def test_nonphysical_state_is_flagged_not_trapped():
    """A negative initial density is reported through the sticky flag and the
    status of pond_status_flags; the context stays usable."""
    n = 16
    rho = np.ones((n, n))
    rho[3, 4] = -0.5
    cfg = W._base(2, n, n, tau=1e-3, dx=1.0 / n, bc=(0, 0, 0, 0))
    cfg["dt"] = 1e-3
    sim = pond.Sim(cfg)
    sim.init(rho, np.zeros((n, n)), np.zeros((n, n)), np.ones((n, n)))
    sim.step(1)
    st, flags, _, _ = sim.flags()
    assert st == pond.POND_E_NONPHYSICAL and flags & pond.POND_FLAG_NONPHYSICAL
    pond.pond_reset_flags(sim.ctx)
    sim.init(np.ones((n, n)), np.zeros((n, n)), np.zeros((n, n)), np.ones((n, n)))
    sim.step(2)
    assert sim.flags()[0] == pond.POND_OK
    sim.close()


def test_step_before_init_and_bad_count():
    cfg = W._base(1, 10, 1, tau=1e-3, dx=0.1)
    cfg["dt"] = 1e-3
    sim = pond.Sim(cfg)
    with pytest.raises(pond.PondError) as e:
        sim.step(1)
    assert e.value.status == pond.POND_E_STATE
    sim.init(np.ones(10), np.zeros(10), np.zeros(10), np.ones(10))
    with pytest.raises(pond.PondError) as e:
        sim.step(-1)
    assert e.value.status == pond.POND_E_INVAL
    sim.close()


def test_moments_match_oracle_moments():
    rho, ux, uy, T = W.random_state_grid(2, 12, 9, seed=3, mach=1.0)
    cfg = W._base(2, 12, 9, tau=5e-3, dx=1 / 12, bc=(1, 1, 1, 1))
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.3)
    ocfg = oracle.Config.from_dict(cfg)
    ost = oracle.run(ocfg, oracle.init(ocfg, rho, ux, uy, T), 2)
    om = oracle.moments(ocfg, ost)
    sim = pond.Sim(cfg)
    sim.init(rho, ux, uy, T)
    sim.step(2)
    gm = sim.moments()
    sim.close()
    for a, b in zip(gm, om):
        assert _rel(a, b) <= TOL


ITER_CASES = [
    # D, nx, ny, bc, prandtl, limiter, mach, iter_tol, iter_max, steps, parity tolerance
    (1, 300, 1, (1, 1, 1, 1), 1.0, 0, 0.5, 1e-12, 10, 3, TOL),
    (1, 253, 1, (0, 0, 0, 0), 0.71, 1, 0.5, 1e-9, 12, 2, TOL),
    (2, 37, 29, (0, 0, 0, 0), 1.0, 0, 0.5, 1e-12, 10, 2, TOL),
    (2, 21, 18, (1, 1, 0, 0), 0.71, 1, 0.5, 1e-9, 12, 2, TOL),
    # a face whose iterates cycle (a node's v_n changes sign between iterates)
    # feeds rounding differences back through every iteration: 40 of them
    # turn the 1e-16 differences of one trace into ~1e-11
    (1, 253, 1, (0, 0, 0, 0), 0.71, 1, 0.5, 1e-9, 40, 2, 1e-10),
]


@pytest.mark.parametrize("case", range(len(ITER_CASES)))
def test_iterated_face_frame_matches_oracle(case):
    """The iterated face frame (option): same state and the same number of
    unconverged face evaluations as the oracle."""
    D, nx, ny, bc, pr, lim, mach, tol, itmax, steps, ptol = ITER_CASES[case]
    rho, ux, uy, T = W.random_state_grid(D, nx, ny, seed=40 + case, mach=mach)
    cfg = W._base(D, nx, ny, tau=5e-3, dx=1.0 / nx, prandtl=pr, limiter=lim, bc=bc,
                  iterative=1, iter_tol=tol, iter_max=itmax)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4)
    ost, got, flags = _run_both(cfg, rho, ux, uy, T, steps)
    _compare(ost, got, D, tol=ptol)
    assert flags[3] == ost.report["noconv_faces"]
    assert bool(flags[1] & pond.POND_FLAG_NOCONV) == bool(ost.report["noconv_faces"])
    # the iteration statistics, exactly
    assert flags[4:] == (ost.report["face_evals"], ost.report["traces"], ost.report["max_traces"])
    assert flags[4] == steps * ((nx + 1) * ny + (nx * (ny + 1) if D == 2 else 0))


def test_iterated_face_frame_sod_matches_oracle():
    """Sod tube at CFL 0.2 with the iterated frame: the discontinuity face
    falls back to its last physical iterate on both sides."""
    w = W.sod_1d(cfl=0.2)
    cfg = dict(w["cfg"], iterative=1, iter_tol=1e-9, iter_max=60)
    ost, got, flags = _run_both(cfg, w["rho"], w["ux"], w["uy"], w["T"], 60)
    _compare(ost, got, 1)
    assert flags[3] == ost.report["noconv_faces"] and flags[3] > 0
    assert flags[4:] == (ost.report["face_evals"], ost.report["traces"], ost.report["max_traces"])


def _window_oracle_interior(cfg, fields, j, k, steps):
    """Oracle run on the (4 steps + 1)^2 window around an interior cell (j, k)
    (at least 2 steps' reach from every boundary): the centre cell depends
    only on cells within 2 per step, whatever the boundary conditions."""
    r = 2 * steps
    sub = [np.ascontiguousarray(a[k - r:k + r + 1, j - r:j + r + 1]) for a in fields]
    c = dict(cfg, nx=2 * r + 1, ny=2 * r + 1, bc=(1, 1, 1, 1))
    ocfg = oracle.Config.from_dict(c)
    st = oracle.run(ocfg, oracle.init(ocfg, *sub), steps)
    return st.f[:, r, r], st.g[:, r, r], st.ux[r, r], st.uy[r, r], st.T[r, r]


def _check_sampled(cfg, fields, got, cells, steps):
    f, g, ux, uy, T = got
    for j, k in cells:
        of, og, oux, ouy, oT = _window_oracle_interior(cfg, fields, int(j), int(k), steps)
        assert _rel(f[:, k, j], of) <= TOL and _rel(g[:, k, j], og) <= TOL
        assert abs(ux[k, j] - oux) <= TOL * max(abs(oux), 1.0)
        assert abs(uy[k, j] - ouy) <= TOL * max(abs(ouy), 1.0)
        assert abs(T[k, j] - oT) <= TOL * oT


def test_riemann_full_size_sampled_cells_match_oracle():
    """The 1024^2 four-quadrant Riemann problem of the benchmark (QE Pr 0.71,
    minmod), FP64, in the benchmark's launch configuration; 2 steps, 16 seeded
    interior cells (including cells on the quadrant interfaces) checked
    against the oracle one by one."""
    w = W.riemann4_2d(n=1024, seed=1)
    fields = (w["rho"], w["ux"], w["uy"], w["T"])
    sim = pond.Sim(w["cfg"])
    sim.init(*fields)
    sim.step(2)
    got = sim.get_state()
    sim.close()
    rng = np.random.default_rng(8)
    cells = [tuple(x) for x in rng.integers(8, 1016, (12, 2))] + [(511, 512), (512, 511), (510, 300), (700, 513)]
    _check_sampled(w["cfg"], fields, got, cells, 2)


def test_batch_full_size_sampled_cells_match_oracle():
    """The benchmark's 64-instance shock-bubble batch in FP64 (persistent,
    autotuned), 2 steps; 3 seeded interior cells in each of 8 members checked
    against the oracle."""
    ws = [W.shock_bubble_2d(seed=s) for s in range(64)]
    b = pond.Batch(2, pond.POND_FP64, 64)
    sims = []
    for w in ws:
        s = pond.Sim(w["cfg"], stream=b.stream)
        s.init(w["rho"], w["ux"], w["uy"], w["T"])
        b.add(s)
        sims.append(s)
    b.step([2] * 64)
    rng = np.random.default_rng(9)
    for i in rng.choice(64, 8, replace=False):
        w = ws[int(i)]
        n = w["cfg"]["nx"]
        got = sims[int(i)].get_state()
        cells = [tuple(x) for x in rng.integers(8, n - 8, (3, 2))]
        _check_sampled(w["cfg"], (w["rho"], w["ux"], w["uy"], w["T"]), got, cells, 2)
    b.close()
    for s in sims:
        s.close()


def test_iterated_and_averaged_frames_agree_when_resolved():
    """Sec. V.D: at moderate CFL on a resolved grid the iterated and the
    averaged face frame give almost the same solution.  Sod tube, 400 cells,
    CFL 0.2: both within 1e-2 of the exact solution in L1 and within 10 % of
    each other; the iteration makes a few traces per face on average."""
    from tests.riemann_exact import solution

    w = W.sod_1d(n=400, cfl=0.2)
    exact = solution((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), w["x"], w["t_end"])[0]
    l1 = {}
    for it in (0, 1):
        sim = pond.Sim(dict(w["cfg"], iterative=it, iter_tol=1e-9, iter_max=40))
        sim.init(w["rho"], w["ux"], w["uy"], w["T"])
        sim.step(w["steps"])
        rho = sim.moments()[0][0]
        ev, tr, mx = sim.iter_stats()
        sim.close()
        l1[it] = float(np.sum(np.abs(rho - exact)) / 400)
        if it:
            assert ev == w["steps"] * 401 and 1.0 < tr / ev < 10.0 and 1 < mx <= 41
        else:
            assert ev == tr == mx == 0
    assert l1[0] < 1e-2 and l1[1] < 1e-2
    assert abs(l1[1] / l1[0] - 1.0) < 0.1, l1


WALL_CASES = [
    # D, nx, ny, bc, prandtl, limiter, grad_k, appc, mach, steps, tile
    (2, 21, 23, (0, 0, 3, 3), 0.71, 0, 0, 0, 0.8, 3, 0),
    (2, 30, 17, (1, 1, 3, 3), 1.0, 1, 1, 1, 1.0, 2, 2),
    (2, 19, 9, (0, 0, 3, 1), 0.5, 0, 0, 0, 0.6, 2, 9),   # one wall, zero gradient opposite
    (2, 12, 30, (0, 0, 3, 3), 0.71, 1, 0, 0, 0.7, 2, 6),
    (1, 64, 1, (3, 3, 0, 0), 0.71, 0, 0, 0, 0.8, 4, 0),
    (1, 33, 1, (3, 1, 0, 0), 1.0, 1, 0, 1, 1.0, 3, 0),
]
# walls: tangential motion only in 2D, resting in 1D, each at its own temperature
WALLS_2D = ((0.0,) * 4, (0.0,) * 4, (0.0, 0.3, 0.0, 0.9), (0.0, -0.2, 0.0, 1.2))
WALLS_1D = ((0.0, 0.0, 0.0, 0.9), (0.0, 0.0, 0.0, 1.2), (0.0,) * 4, (0.0,) * 4)


@pytest.mark.parametrize("case", range(len(WALL_CASES)))
def test_walls_match_oracle(case):
    """Wall ghosts (reflection plus Chapman-Enskog non-equilibrium) and the
    mean trace at v_n = 0 that walls at rest produce: same state as the
    oracle."""
    D, nx, ny, bc, pr, lim, gk, appc, mach, steps, tile = WALL_CASES[case]
    # T_B < 2 T_w everywhere, so that every reflected ghost temperature is positive
    rho, ux, uy, T = W.random_state_grid(D, nx, ny, seed=90 + case, mach=mach, T=(0.7, 1.4))
    cfg = W._base(D, nx, ny, tau=5e-3, dx=1.0 / nx, prandtl=pr, limiter=lim, grad_k=gk,
                  flux_appc=appc, bc=bc, inflow=WALLS_2D if D == 2 else WALLS_1D)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4)
    ost, got, flags = _run_both(cfg, rho, ux, uy, T, steps, tile=tile)
    _compare(ost, got, D)
    assert flags[1] & pond.POND_FLAG_NONPHYSICAL == 0


def test_walls_are_rejected_where_not_supported():
    bad = [(2, (3, 3, 0, 0)), (2, (2, 1, 3, 3)), (1, (0, 0, 3, 3))]
    for D, bc in bad:
        cfg = W._base(D, 16, 16, tau=5e-3, dx=1.0 / 16, bc=bc, dt=1e-3)
        with pytest.raises(pond.PondError):
            pond.Sim(cfg)


@pytest.mark.parametrize("prandtl", [0.7])
def test_thermal_couette_at_the_papers_size(prandtl):
    """Sec. V.B.2: L = 150 cells, Ma 0.5, Re 100, T_C = 1, Ec 20, from the
    analytic steady state run for a quarter of the viscous time L^2/nu: the
    temperature stays within 1.5 % of the analytic profile's height (the
    wall reflection's first-order error) and the velocity profile linear."""
    w = W.thermal_couette_2d(ny=150, nx=8, prandtl=prandtl, ec=20.0, re=100.0)
    steps = int(0.25 * (100.0 / w["u0"]) / w["cfg"]["dt"])
    sim = pond.Sim(w["cfg"])
    sim.init(w["rho"], w["ux"], w["uy"], w["T"])
    sim.step(steps)
    m = sim.moments()
    flags = sim.flags()
    sim.close()
    assert flags[1] == 0
    theta = (m[3][:, 3] - w["t_cold"]) / w["dT"]
    exact = w["theta"](w["y"])
    assert np.max(np.abs(theta - exact)) / np.max(exact) < 0.015
    assert np.max(np.abs(m[1][:, 3] / w["u0"] - w["y"])) < 1e-3
    assert np.max(np.abs(m[3] - m[3][:, :1])) < 1e-12  # uniform along the walls


Q5_CASES = [
    # nx, ny, bc, prandtl, limiter, grad_k, appc, mach, steps, iterative
    (19, 17, (0, 0, 0, 0), 1.0, 0, 0, 0, 0.8, 2, 0),
    (21, 18, (1, 1, 1, 1), 0.71, 1, 0, 0, 1.0, 2, 0),
    (17, 23, (2, 1, 1, 1), 1.0, 0, 1, 0, 0.6, 2, 0),
    (20, 19, (0, 0, 1, 1), 0.71, 0, 0, 1, 1.0, 2, 0),
    (18, 16, (0, 0, 3, 3), 0.71, 1, 0, 0, 0.7, 2, 0),
    (16, 17, (0, 0, 0, 0), 1.0, 0, 0, 0, 0.5, 2, 1),
]


def test_d2q25_tiles_compute_the_same_step():
    """The two D2Q25 tile shapes (8x8 with 128 threads and two CTAs per SM,
    the default; 8x8 with 160 threads and one CTA): the same state to
    rounding."""
    nx, ny = 37, 29
    rho, ux, uy, T = W.random_state_grid(2, nx, ny, seed=141, mach=0.8, T=(0.7, 1.4))
    cfg = W._base(2, nx, ny, qf=5, tau=5e-3, dx=1.0 / nx, prandtl=0.71, bc=(1, 1, 1, 1))
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4, c_max=W.C_MAX_D1Q5)
    out = {}
    for tile in (2, 10):
        sim = pond.Sim(dict(cfg, tile=tile))
        sim.init(rho, ux, uy, T)
        sim.step(3)
        out[tile] = sim.get_state()
        assert sim.info()[2] == tile
        sim.close()
    for a, b in zip(out[2], out[10]):
        assert _rel(a, b) <= 1e-13


@pytest.mark.parametrize("case", range(len(Q5_CASES)))
def test_d2q25_matches_oracle(case):
    """The D2Q25 f-lattice (D1Q5 per axis, fourth-order invariance) with D2Q9
    for g: the same state as the oracle, across boundaries, QE, limiters,
    Grad-K of total order 4, Appendix C, walls and the iterated frame."""
    nx, ny, bc, pr, lim, gk, appc, mach, steps, it = Q5_CASES[case]
    rho, ux, uy, T = W.random_state_grid(2, nx, ny, seed=130 + case, mach=mach, T=(0.7, 1.4))
    cfg = W._base(2, nx, ny, qf=5, tau=5e-3, dx=1.0 / nx, prandtl=pr, limiter=lim, grad_k=gk,
                  flux_appc=appc, bc=bc, iterative=it, iter_tol=1e-10, iter_max=12,
                  inflow=WALLS_2D if 3 in bc else ((1.1, 0.5, -0.2, 0.8),) * 4)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4, c_max=W.C_MAX_D1Q5)
    ost, got, flags = _run_both(cfg, rho, ux, uy, T, steps)
    assert got[0].shape[0] == 25
    _compare(ost, got, 2)
    assert flags[1] & pond.POND_FLAG_NONPHYSICAL == 0
    if it:
        assert flags[4:] == (ost.report["face_evals"], ost.report["traces"], ost.report["max_traces"])


@pytest.mark.parametrize("precision,D", [(pond.POND_FP64, 2), (pond.POND_FP32_MIXED, 2),
                                         (pond.POND_FP64, 1)])
def test_strips_give_the_same_state_bit_for_bit(precision, D):
    """A CTA steps a strip of tiles and hands each tile's right-edge x-faces
    to the next: every strip length must give the state of one tile per CTA,
    bit for bit (ragged last tiles in x and y, zero-gradient and walled
    sides)."""
    nx, ny = (250, 61) if D == 2 else (2000, 1)
    rho, ux, uy, T = W.random_state_grid(D, nx, ny, seed=81, mach=0.4, T=(0.8, 1.3))
    if D == 2:
        walls = ((0.0,) * 4, (0.0,) * 4, (0.0, 0.2, 0.0, 1.0), (0.0, -0.1, 0.0, 1.1))
        cfg = W._base(2, nx, ny, tau=5e-3, dx=1.0 / nx, prandtl=0.71, bc=(1, 1, 3, 3), inflow=walls)
    else:
        cfg = W._base(1, nx, 1, tau=5e-3, dx=1.0 / nx, prandtl=0.71, bc=(1, 1, 1, 1))
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4)
    ref = None
    for strip in (1, 2, 3, 8):
        sim = pond.Sim(dict(cfg, precision=precision, strip=strip))
        sim.init(rho, ux, uy, T)
        sim.step(3)
        st = sim.get_state()
        flags = sim.flags()[1]
        sim.close()
        assert flags & pond.POND_FLAG_NONPHYSICAL == 0, strip
        if ref is None:
            ref = st
        for a, b in zip(st, ref):
            assert np.array_equal(a, b), strip


def test_strip_of_three_matches_oracle():
    """Strips of three tiles on a ragged periodic / inflow grid: the handed-over
    faces give the oracle's state."""
    rho, ux, uy, T = W.random_state_grid(2, 53, 37, seed=83, mach=1.0)
    cfg = W._base(2, 53, 37, tau=5e-3, dx=1.0 / 53, prandtl=0.71, limiter=1, bc=(2, 1, 0, 0),
                  inflow=((1.1, 0.5, -0.2, 0.8),) * 4)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.4)
    ost, got, flags = _run_both(dict(cfg, strip=3), rho, ux, uy, T, 2)
    _compare(ost, got, 2)
