"""Step-level pins of the oracle: an independent multi-precision restatement on
tiny grids, exact conservation (Appendix C), uniform flow, mirror symmetry,
the exact Riemann solution of the Sod problem, and second-order convergence
on a smooth advected pulse."""
import math

import numpy as np
import pytest

import oracle
from paper_2302_00310_gb300 import workloads as W
from tests import riemann_exact
from tests.restate_step import Restated

GAMMA = 1.4


def _state(cfg_d, rho, ux, uy, T):
    cfg = oracle.Config.from_dict(cfg_d)
    return cfg, oracle.init(cfg, rho, ux, uy, T)


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def _random_nonequilibrium(cfg, st, seed, amp=0.05):
    """Perturb the populations of an equilibrium state and bring each cell back
    into its co-moving frame (so the step starts from a non-equilibrium,
    co-moving state)."""
    rng = np.random.default_rng(seed)
    st = st.copy()
    st.f *= 1 + amp * rng.uniform(-1, 1, st.f.shape)
    st.g *= 1 + amp * rng.uniform(-1, 1, st.g.shape)
    ny, nx = st.T.shape
    for k in range(ny):
        for j in range(nx):
            m, ok = oracle.macro(cfg.qf, cfg.qg, cfg.D, cfg.gamma, st.f[:, k, j], st.g[:, k, j],
                                 (st.ux[k, j], st.uy[k, j]), st.T[k, j])
            assert ok
            un = m[1:1 + cfg.D]
            st.f[:, k, j] = oracle.transform(cfg.qf, cfg.D, st.f[:, k, j], (st.ux[k, j], st.uy[k, j])[:cfg.D],
                                             st.T[k, j], un, m[3])
            st.g[:, k, j] = oracle.transform(cfg.qg, cfg.D, st.g[:, k, j], (st.ux[k, j], st.uy[k, j])[:cfg.D],
                                             st.T[k, j], un, m[3])
            st.ux[k, j], st.T[k, j] = m[1], m[3]
            if cfg.D == 2:
                st.uy[k, j] = m[2]
    return st


CASES = [
    # D, nx, ny, bc, prandtl, limiter, mach
    (1, 6, 1, (1, 1, 1, 1), 1.0, 0, 0.8),
    (1, 6, 1, (0, 0, 0, 0), 0.71, 1, 1.5),
    (1, 5, 1, (2, 1, 1, 1), 1.0, 0, 0.5),
    (2, 4, 4, (0, 0, 0, 0), 1.0, 0, 0.7),
    (2, 4, 3, (1, 1, 0, 0), 0.71, 1, 1.2),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_oracle_step_matches_multiprecision_restatement(case):
    mp = pytest.importorskip("mpmath")
    D, nx, ny, bc, pr, lim, mach = CASES[case]
    rho, ux, uy, T = W.random_state_grid(D, nx, ny, seed=100 + case, mach=mach)
    d = W._base(D, nx, ny, tau=2e-3, dx=1.0 / nx, prandtl=pr, limiter=lim, bc=bc,
                inflow=((1.2, 0.4, 0.1, 0.9),) * 4)
    d["dt"] = W.dt_from_cfl(ux, uy, T, d["dx"], 0.4)
    cfg, st = _state(d, rho, ux, uy, T)
    st = _random_nonequilibrium(cfg, st, seed=case)
    out = oracle.run(cfg, st, 1)
    R = Restated(mp, d, dps=30)
    ref = R.to_arrays(R.step(R.from_arrays(st.f, st.g, st.ux, st.uy, st.T)))
    for got, want in zip((out.f, out.g, out.ux, out.uy, out.T), ref):
        assert _rel(got, want) < 1e-12 or np.max(np.abs(got - want)) < 1e-13


@pytest.mark.parametrize("grad_k,appc,pr", [(0, 0, 1.0), (1, 0, 1.0), (0, 1, 1.0), (0, 0, 0.71), (1, 1, 0.5)])
def test_conservation_on_periodic_grid(grad_k, appc, pr):
    """Total mass, momentum and energy are conserved to rounding (Appendix C).
    dt/tau < 1 here: the explicit quasi-equilibrium half steps of Sec. IV.B
    amplify third-order modes by (1 + dt/(2 tau) (1 - Pr))^2 per step, which
    the BGK factor (2 tau - dt)/(2 tau + dt) no longer offsets at dt/tau >> 1."""
    D, n = 2, 8
    rho, ux, uy, T = W.random_state_grid(D, n, n, seed=7, mach=1.0)
    d = W._base(D, n, n, tau=2e-2, dx=1.0 / n, prandtl=pr, grad_k=grad_k, flux_appc=appc,
                bc=(0, 0, 0, 0))
    d["dt"] = W.dt_from_cfl(ux, uy, T, d["dx"], 0.3)
    cfg, st = _state(d, rho, ux, uy, T)

    def totals(s):
        m = oracle.moments(cfg, s)
        r, vx, vy, t = m
        return np.array([r.sum(), (r * vx).sum(), (r * vy).sum(),
                         (r * t / (GAMMA - 1) + 0.5 * r * (vx**2 + vy**2)).sum()])

    t0 = totals(st)
    out = oracle.run(cfg, st, 20)
    t1 = totals(out)
    scale = np.array([t0[0], t0[0], t0[0], t0[3]])
    assert np.max(np.abs(t1 - t0) / scale) < 1e-13
    assert out.report["flags"] == 0


@pytest.mark.parametrize("D", [1, 2])
def test_uniform_flow_stays_uniform(D):
    """A uniform state at Mach 5 stays uniform (every face sees identical data)."""
    n = 6
    cs = math.sqrt(GAMMA * 0.7)
    shp = (n if D == 2 else 1, n)
    rho, T = np.full(shp, 1.3), np.full(shp, 0.7)
    ux, uy = np.full(shp, 5 * cs * 0.8), np.full(shp, (5 * cs * 0.6) if D == 2 else 0.0)
    d = W._base(D, n, n, tau=1e-3, dx=1.0 / n, bc=(0, 0, 0, 0))
    d["dt"] = W.dt_from_cfl(ux, uy, T, d["dx"], 0.5)
    cfg, st = _state(d, rho, ux, uy, T)
    out = oracle.run(cfg, st, 10)
    np.testing.assert_allclose(out.f, st.f, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(out.ux, st.ux, rtol=1e-13)
    np.testing.assert_allclose(out.T, st.T, rtol=1e-13)


@pytest.mark.parametrize("pr,lim", [(1.0, 0), (0.71, 1)])
def test_mirror_symmetry_of_config3(pr, lim):
    """Riemann configuration 3 is symmetric under x <-> y (Sec. V.A.3); so must
    the solution be, with u_x and u_y exchanged and the populations transposed.
    (tau raised so that dt/tau ~ 1 on this coarse grid.)"""
    w = W.config3_2d(n=12, prandtl=pr)
    w["cfg"]["tau"], w["cfg"]["limiter"] = 5e-3, lim
    cfg, st = _state(w["cfg"], w["rho"], w["ux"], w["uy"], w["T"])
    out = oracle.run(cfg, st, 4)
    assert out.report["flags"] == 0
    np.testing.assert_allclose(out.T, out.T.T, rtol=1e-12)
    np.testing.assert_allclose(out.ux, out.uy.T, rtol=1e-12, atol=1e-14)
    fq = out.f.reshape(4, 4, 12, 12)  # [iy, ix, y, x]
    np.testing.assert_allclose(fq, np.transpose(fq, (1, 0, 3, 2)), rtol=1e-11, atol=1e-14)


def test_reflection_symmetry_1d():
    """x -> 1 - x with u -> -u maps a tube onto its mirror image."""
    w = W.tube_1d(40, (1.0, 0.3, 1.0), (0.3, -0.2, 0.4), tau=1e-3, cfl=0.3)
    cfg, st = _state(w["cfg"], w["rho"], w["ux"], w["uy"], w["T"])
    wm = W.tube_1d(40, (0.3, 0.2, 0.4), (1.0, -0.3, 1.0), tau=1e-3, cfl=0.3)
    wm["cfg"]["dt"] = w["cfg"]["dt"]
    cfgm, stm = _state(wm["cfg"], wm["rho"], wm["ux"], wm["uy"], wm["T"])
    a = oracle.run(cfg, st, 15)
    b = oracle.run(cfgm, stm, 15)
    np.testing.assert_allclose(a.T[0], b.T[0][::-1], rtol=1e-12)
    np.testing.assert_allclose(a.ux[0], -b.ux[0][::-1], rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(a.f[:, 0, :], b.f[::-1, 0, ::-1], rtol=1e-11, atol=1e-14)


def _sod_l1(cfl):
    w = W.sod_1d(cfl=cfl)
    cfg, st = _state(w["cfg"], w["rho"], w["ux"], w["uy"], w["T"])
    out = oracle.run(cfg, st, w["steps"])
    rho = oracle.moments(cfg, out)[0, 0]
    ex = riemann_exact.solution((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), w["x"], w["t_end"])
    return np.mean(np.abs(rho - ex[0])), out.report


def test_exact_riemann_solver_star_state():
    """The test-side exact solver reproduces the classical Sod star state."""
    p, u = riemann_exact.star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(p - 0.30313) < 1e-5 and abs(u - 0.92745) < 1e-5


@pytest.mark.parametrize("cfl", [None, 0.2])
def test_sod_density_within_l1_of_exact_solution(cfl):
    """Sod tube at t = 0.2 on 400 cells: L1(rho) against the exact Riemann
    solution; config time step (CFL ~ 0.75-1.1) and the paper's CFL 0.2."""
    l1, rep = _sod_l1(cfl)
    assert rep["flags"] == 0
    assert l1 < 1e-2, l1


def test_pulse_second_order_convergence_1d():
    """Periodic isobaric pulse advected at Mach 2 (an Euler entropy wave: exact
    solution = translated profile).  L1 error falls at ~2nd order (Sec. V.B.1)."""
    errs = []
    U, t_end, sigma, amp = 2 * math.sqrt(GAMMA), 0.1, 0.1, 0.1
    for n in (50, 100, 200):
        x = (np.arange(n) + 0.5) / n
        prof = lambda xx: sum(np.exp(-((xx - 0.5 - s) ** 2) / (2 * sigma**2)) for s in (-1, 0, 1))
        rho = 1 + amp * prof(x)
        d = W._base(1, n, 1, tau=1e-6, dx=1.0 / n, bc=(0, 0, 0, 0))
        d["dt"] = W.dt_from_cfl(np.full(n, U), 0 * x, 1 / rho, 1.0 / n, 0.2)
        steps = int(math.ceil(t_end / d["dt"]))
        d["dt"] = t_end / steps
        cfg, st = _state(d, rho, np.full(n, U), 0 * x, 1 / rho)
        out = oracle.run(cfg, st, steps)
        r = oracle.moments(cfg, out)[0, 0]
        exact = 1 + amp * prof((x - U * t_end) % 1.0)
        errs.append(np.mean(np.abs(r - exact)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.5, (errs, orders)


@pytest.mark.slow
def test_pulse_second_order_convergence_2d():
    """The 2D periodic isobaric pulse (Mach 2 at 30 degrees, sigma 0.15) to
    t = 0.05 at 24^2, 48^2, 96^2 against the translated profile (the exact
    Euler entropy wave; tau = 1e-6 keeps the viscous change of the profile far
    below the discretisation error).  L1 falls at ~2nd order (Sec. V.B.1)."""
    errs = []
    t_end = 0.05
    for n in (24, 48, 96):
        w = W.pulse_2d(n=n, seed=0, sigma=0.15, centre=(0.5, 0.5), tau=1e-6)
        d = dict(w["cfg"])
        steps = int(math.ceil(t_end / d["dt"]))
        d["dt"] = t_end / steps
        cfg, st = _state(d, w["rho"], w["ux"], w["uy"], w["T"])
        r = oracle.moments(cfg, oracle.run(cfg, st, steps))[0]
        errs.append(np.mean(np.abs(r - W.pulse_exact_2d(w, t_end))))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.5, (errs, orders)


def test_1d_inflow_ghost_has_no_uy():
    """A 1D state has no u_y (the 1D model of Sec. V): the inflow's u_y slot
    must not reach the boundary face's frame or its energy sum."""
    rho, ux, uy, T = W.random_state_grid(1, 12, 1, seed=4, mach=0.8)
    out = []
    for vy in (0.0, 0.7):
        d = W._base(1, 12, 1, tau=2e-3, dx=1.0 / 12, bc=(2, 2, 0, 0), inflow=((1.1, 0.3, vy, 0.9),) * 4)
        d["dt"] = W.dt_from_cfl(ux, uy, T, d["dx"], 0.4)
        cfg = oracle.Config.from_dict(d)
        out.append(oracle.run(cfg, oracle.init(cfg, rho, ux, uy, T), 3))
    assert np.array_equal(out[0].f, out[1].f) and np.array_equal(out[0].T, out[1].T)
