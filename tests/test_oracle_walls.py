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
