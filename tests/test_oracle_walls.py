"""Wall boundaries of the oracle (Sec. IV.D): reflected ghost cells carrying
the Chapman-Enskog non-equilibrium, pinned by

* a resting uniform gas between resting walls at its own temperature: the
  ghosts reproduce it and nothing moves;
* mirror symmetry: a state symmetric about the channel's mid-plane between two
  equal walls stays symmetric (the two walls' index arithmetic agree);
* the thermal Couette flow of Sec. V.B.2 against its analytic temperature
  profile (T - T_C)/(T_H - T_C) = y + Pr Ec/2 y (1 - y): the velocity profile
  is linear to 1e-3, and the temperature error falls at first order under
  refinement.  The reflection T_G = 2 T_w - T_B puts the wall value at the
  mid-point, but the wall-face gradient (T_0 - T_G)/dx = T' + dx/4 T'' + ...
  carries a first-order error where the profile is curved (the viscous
  heating makes T'' = -Pr Ec dT), so the error halves when dx halves.
"""
import numpy as np
import pytest

import oracle
from paper_2302_00310_gb300 import workloads as W


def _moments(cfg, st):
    return oracle.moments(oracle.Config.from_dict(cfg), st)


@pytest.mark.parametrize("D", [1, 2])
def test_resting_gas_between_resting_walls_stays_at_rest(D):
    n = 12
    shp = (n if D == 2 else 1, n)
    rho, T = np.full(shp, 1.3), np.full(shp, 0.9)
    z = np.zeros(shp)
    bc = (0, 0, 3, 3) if D == 2 else (3, 3, 0, 0)
    wall = (0.0, 0.0, 0.0, 0.9)
    cfg = W._base(D, n, n, tau=5e-3, dx=1.0 / n, prandtl=0.71, bc=bc, inflow=(wall,) * 4)
    cfg["dt"] = W.dt_from_cfl(z, z, T, cfg["dx"], 0.3)
    oc = oracle.Config.from_dict(cfg)
    st0 = oracle.init(oc, rho, z, z, T)
    st = oracle.run(oc, st0, 20)
    np.testing.assert_allclose(st.f, st0.f, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(st.g, st0.g, rtol=1e-13, atol=1e-15)
    assert np.max(np.abs(st.ux)) < 1e-14 and np.max(np.abs(st.uy)) < 1e-14
    np.testing.assert_allclose(st.T, T, rtol=1e-13)


def test_mirror_symmetric_channel_stays_symmetric():
    nx, ny = 6, 10
    g = W.rng(3)
    rho = g.uniform(0.8, 1.2, (ny // 2, nx))
    T = g.uniform(0.8, 1.2, (ny // 2, nx))
    ux = g.uniform(-0.3, 0.3, (ny // 2, nx))
    uy = g.uniform(-0.3, 0.3, (ny // 2, nx))
    # reflect about the mid-plane y = 1/2: rho, T, ux even, uy odd
    rho, T, ux = (np.vstack([a, a[::-1]]) for a in (rho, T, ux))
    uy = np.vstack([uy, -uy[::-1]])
    wall = (0.0, 0.1, 0.0, 1.05)
    cfg = W._base(2, nx, ny, tau=5e-3, dx=1.0 / ny, prandtl=0.71, bc=(0, 0, 3, 3),
                  inflow=(wall,) * 4)
    cfg["dt"] = W.dt_from_cfl(ux, uy, T, cfg["dx"], 0.3)
    oc = oracle.Config.from_dict(cfg)
    st = oracle.run(oc, oracle.init(oc, rho, ux, uy, T), 6)
    m = _moments(cfg, st)
    for field, sign in zip(m, (1, 1, -1, 1)):
        np.testing.assert_allclose(field, sign * field[::-1], rtol=1e-12, atol=1e-13)
    assert np.max(np.abs(m[2])) > 1e-4  # the case is not trivially at rest


def _couette_error(ny, prandtl, steps):
    w = W.thermal_couette_2d(ny=ny, nx=2, prandtl=prandtl)
    oc = oracle.Config.from_dict(w["cfg"])
    st = oracle.run(oc, oracle.init(oc, w["rho"], w["ux"], w["uy"], w["T"]), steps)
    assert st.report["flags"] == 0
    m = _moments(w["cfg"], st)
    theta = (m[3][:, 0] - w["t_cold"]) / w["dT"]
    exact = w["theta"](w["y"])
    u_err = np.max(np.abs(m[1][:, 0] / w["u0"] - w["y"]))
    return np.max(np.abs(theta - exact)) / np.max(exact), u_err


@pytest.mark.slow
def test_thermal_couette_matches_the_analytic_profile_at_first_order():
    # steady from the analytic start after about one viscous time L^2 / nu
    e16, u16 = _couette_error(16, 1.0, 8000)
    e32, u32 = _couette_error(32, 1.0, 16000)
    assert u16 < 1e-3 and u32 < 1e-3
    assert e16 < 0.06
    assert 0.35 < e32 / e16 < 0.65, (e16, e32)
    # a lower Prandtl number halves the heating term Pr Ec / 2
    e16b, _ = _couette_error(16, 0.5, 8000)
    assert e16b < 0.06


# ---- the ghost's Chapman-Enskog moments, recovered by quadrature ------------
def _ghost_moments(q, D, pops, T):
    """Central moments of a ghost's populations in its co-moving frame: the
    nodes are xi_i = sqrt(T) c_i (node i = iy*q + ix).  Returns the moments of
    order 0..3 as arrays over the D axes."""
    c = np.polynomial.hermite_e.hermegauss(q)[0]  # the roots of He_q, ascending (Table I)
    if D == 1:
        xi = np.sqrt(T) * c[:, None]
    else:
        xi = np.sqrt(T) * np.array([[c[i % q], c[i // q]] for i in range(q * q)])
    m0 = pops.sum()
    m1 = np.einsum("i,ia->a", pops, xi)
    m2 = np.einsum("i,ia,ib->ab", pops, xi, xi)
    m3 = np.einsum("i,ia,ib,ic->abc", pops, xi, xi, xi)
    return m0, m1, m2, m3


@pytest.mark.parametrize("D", [1, 2])
def test_wall_ghost_carries_the_chapman_enskog_moments_of_sec_iv_d(D):
    """Linear fields u = u_0 + a y (+ e y along the normal in 2D), T = T_0 + b y
    with the walls on the same lines: the ghost's centred gradients are exactly
    (a, e, b).  Its populations, summed by quadrature in its co-moving frame,
    must carry the equilibrium plus the paper's first-order non-equilibrium
    (Sec. IV.D) scaled by 1 + dt/(2 tau_1) (the stored variable is phi~):
        P^(1)  = -tau_1 rho T (S - (div u)/C_v I)
        Q^(1)  = -tau_2 rho T sym(grad T I)              (central: no u P^(1) part)
        M_g0   = -tau_1 rho T (2 C_v - D) (div u)/C_v
        M_g1   = -tau_2 rho T (2 C_v - D) grad T          (central: no M_g0 u part)
        M_g2   = -tau_1 rho T (2 C_v - D) T S             (the T S term only)
    with S = grad u + grad u^T.  Pr = 0.5 makes tau_2 = 2 tau_1 and
    dt = tau_1 makes the factor 1.5, so a swapped relaxation time or a missing
    factor changes every checked moment by a third or more."""
    tau, pr, gamma = 5e-3, 0.5, 1.4
    t1, t2, cv = tau, tau / pr, 1.0 / (gamma - 1.0)
    dt = tau
    cf = 1.0 + dt / (2.0 * t1)
    rho0, u0, a, e, T0, b = 1.3, 0.3, 0.8, 0.5, 0.9, 0.4
    n = 6
    dx = 1.0 / n
    y = (np.arange(n) + 0.5) * dx
    if D == 2:
        nx = 4
        shp = (n, nx)
        Y = np.repeat(y[:, None], nx, axis=1)
        ux, uy, T = u0 + a * Y, e * Y, T0 + b * Y
        walls = ((0.0,) * 4, (0.0,) * 4, (0.0, u0, 0.0, T0), (0.0, u0 + a, e, T0 + b))
        cfg = W._base(2, nx, n, tau=tau, dx=dx, prandtl=pr, gamma=gamma, bc=(0, 0, 3, 3), inflow=walls)
        gj, gk = 1, -1
    else:
        shp = (1, n)
        ux, uy, T = (u0 + a * y)[None, :], np.zeros(shp), (T0 + b * y)[None, :]
        walls = ((0.0, u0, 0.0, T0), (0.0, u0 + a, 0.0, T0 + b), (0.0,) * 4, (0.0,) * 4)
        cfg = W._base(1, n, 1, tau=tau, dx=dx, prandtl=pr, gamma=gamma, bc=(3, 3, 0, 0), inflow=walls)
        gj, gk = -1, 0
    cfg["dt"] = dt
    oc = oracle.Config.from_dict(cfg)
    st = oracle.init(oc, np.full(shp, rho0), ux, uy, T)
    f, g, (gux, guy, gT) = oracle.ghost(oc, st, gj, gk)

    # the ghost's fields: the linear continuation half a cell beyond the wall
    yg = -0.5 * dx
    assert gT == pytest.approx(T0 + b * yg, rel=1e-14)
    assert gux == pytest.approx(u0 + a * yg, rel=1e-14)
    if D == 2:
        assert guy == pytest.approx(e * yg, abs=1e-15)
    rho, Tg = rho0, gT
    # exact gradients: grad u[d][c] = d u_c / d x_d, grad T[d]
    if D == 2:
        gu = np.array([[0.0, 0.0], [a, e]])
        gTv = np.array([0.0, b])
        u = np.array([gux, guy])
    else:
        gu = np.array([[a]])
        gTv = np.array([b])
        u = np.array([gux])
    I = np.eye(D)
    div = np.trace(gu)
    S = gu + gu.T
    rT = rho * Tg
    P1 = -t1 * rT * (S - div / cv * I)
    Q1 = -t2 * rT * (np.einsum("a,bc->abc", gTv, I) + np.einsum("b,ac->abc", gTv, I)
                     + np.einsum("c,ab->abc", gTv, I))
    gf = 2.0 * cv - D
    Mg0 = -t1 * rT * gf * div / cv
    Mg1 = -t2 * rT * gf * gTv
    Mg2 = -t1 * rT * gf * Tg * S

    m0, m1, m2, m3 = _ghost_moments(oc.qf, D, f, Tg)
    scale = rT * (abs(a) + abs(b)) * tau
    assert m0 == pytest.approx(rho, rel=1e-13)
    np.testing.assert_allclose(m1, 0.0, atol=1e-13 * rho)
    np.testing.assert_allclose(m2, rT * I + cf * P1, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(m3, cf * Q1, rtol=0, atol=1e-12 * scale)

    geq0 = (cv - 0.5 * D) * Tg * rho
    n0, n1, n2, _ = _ghost_moments(oc.qg, D, g, Tg)
    assert n0 - geq0 == pytest.approx(cf * Mg0, abs=1e-12 * scale)
    np.testing.assert_allclose(n1, cf * Mg1, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(n2 - geq0 * Tg * I, cf * Mg2, rtol=0, atol=1e-12 * scale)
    # the reading of M_g2 on its own: the printed form's extra term
    # sym(u grad T) is not carried (it is not the raw form of a central moment
    # that the frame change would produce), and here it would be visible
    extra = -t1 * rT * gf * (np.outer(u, gTv) + np.outer(gTv, u))
    assert np.max(np.abs(extra)) > 0.1 * np.max(np.abs(Mg2))
    assert not np.allclose(n2 - geq0 * Tg * I, cf * (Mg2 + extra), rtol=1e-3, atol=0)
