"""The D2Q25 f-lattice (Table I: five Gauss-Hermite nodes per axis, the roots
of He_5; Sec. II.D.2: frame-invariant moments to fourth order per axis) in the
oracle, with D2Q9 for g as in every run of the paper.  Pins:

* Table I's D1Q5 weights reproduce the Gaussian moments to degree 9;
* the transformation equals Appendix B's matrix form M(lambda')^-1 M(lambda)
  solved in 50-digit arithmetic, in 2D;
* fourth-order invariance: the fourth moment of rho G W in any frame is the
  Maxwellian one, rho (u^4 + 6 u^2 T + 3 T^2) per axis, so the deviation R'
  of Eq. DeviationR, which D2Q16 leaves, vanishes;
* conservation of mass, momentum and energy on a periodic grid, and a
  uniform Mach-3 flow staying uniform, over whole steps.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2302_00310_gb300 import workloads as W

GAMMA = 1.4


def test_d1q5_weights_reproduce_gaussian_moments():
    c, w, _ = oracle.lattice(5)
    for k, want in ((0, 1.0), (2, 1.0), (4, 3.0), (6, 15.0), (8, 105.0)):
        assert abs(np.sum(w * c**k) - want) < 1e-12 * want
    for k in (1, 3, 5, 7, 9):
        assert abs(np.sum(w * c**k)) < 1e-12


@pytest.mark.parametrize("fr", range(3))
def test_d2q25_transform_equals_appendix_b_matrix_form(fr):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    frames = [((0.3, -0.2), 1.0, (0.1, 0.4), 1.3), ((2.4, 1.3), 0.7, (1.9, 1.0), 0.9),
              ((-1.0, 0.5), 2.0, (0.0, 0.0), 1.0)]
    u, T, up, Tp = frames[fr]
    f = np.random.default_rng(11 + fr).uniform(0.1, 1.0, 25)
    got = oracle.transform(5, 2, f, u, T, up, Tp)
    c, _, _ = oracle.lattice(5)
    cm = [mp.mpf(float(x)) for x in c]

    def M(u, T):
        sT = mp.sqrt(mp.mpf(T))
        v = [(sT * cm[j % 5] + mp.mpf(u[0]), sT * cm[j // 5] + mp.mpf(u[1])) for j in range(25)]
        m = mp.matrix(25, 25)
        for r, (a, b) in enumerate((a, b) for a in range(5) for b in range(5)):
            for j, (vx, vy) in enumerate(v):
                m[r, j] = vx**a * vy**b
        return m

    rhs = M(u, T) * mp.matrix([mp.mpf(float(x)) for x in f])
    want = np.array([float(x) for x in mp.lu_solve(M(up, Tp), rhs)])
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.abs(f).sum())


@pytest.mark.parametrize("q", [4, 5])
def test_fourth_moment_of_a_moved_equilibrium(q):
    """rho G W in a foreign frame: its fourth moment along x is the
    Maxwellian rho (u^4 + 6 u^2 T + 3 T^2) on D2Q25; on D2Q16 the deviation
    -rho (xi^4 + 6 theta xi^2 + 3 theta^2) of Eq. DeviationR remains."""
    rho, u, T, up, Tp = 1.3, (0.7, -0.4), 0.9, (0.2, 0.3), 1.4
    c, w, _ = oracle.lattice(q)
    W2 = np.outer(w, w).ravel()  # [iy][ix] flattened, x fastest
    feq = oracle.transform(q, 2, rho * W2, u, T, up, Tp)
    cx = np.tile(c, q)
    vx = up[0] + math.sqrt(Tp) * cx
    m4 = float(np.sum(feq * vx**4))
    maxw = rho * (u[0] ** 4 + 6 * u[0] ** 2 * T + 3 * T**2)
    if q == 5:
        assert abs(m4 - maxw) < 1e-12 * maxw
    else:
        xi, th = u[0] - up[0], T - Tp
        assert abs(m4 - maxw + rho * (xi**4 + 6 * th * xi**2 + 3 * th**2)) < 1e-12 * maxw


@pytest.mark.parametrize("grad_k,pr", [(0, 1.0), (1, 0.71)])
def test_d2q25_conserves_on_a_periodic_grid(grad_k, pr):
    n = 8
    rho, ux, uy, T = W.random_state_grid(2, n, n, seed=17, mach=1.0)
    d = W._base(2, n, n, qf=5, tau=2e-2, dx=1.0 / n, prandtl=pr, grad_k=grad_k, bc=(0, 0, 0, 0))
    d["dt"] = W.dt_from_cfl(ux, uy, T, d["dx"], 0.3, c_max=W.C_MAX_D1Q5)
    cfg = oracle.Config.from_dict(d)
    st = oracle.init(cfg, rho, ux, uy, T)

    def totals(s):
        r, vx, vy, t = oracle.moments(cfg, s)
        return np.array([r.sum(), (r * vx).sum(), (r * vy).sum(),
                         (r * t / (GAMMA - 1) + 0.5 * r * (vx**2 + vy**2)).sum()])

    t0 = totals(st)
    out = oracle.run(cfg, st, 12)
    t1 = totals(out)
    assert out.report["flags"] == 0
    assert np.max(np.abs(t1 - t0) / np.array([t0[0], t0[0], t0[0], t0[3]])) < 1e-13


def test_d2q25_uniform_flow_stays_uniform():
    n = 6
    cs = math.sqrt(GAMMA * 0.7)
    rho, T = np.full((n, n), 1.3), np.full((n, n), 0.7)
    ux, uy = np.full((n, n), 3 * cs * 0.8), np.full((n, n), 3 * cs * 0.6)
    d = W._base(2, n, n, qf=5, tau=1e-3, dx=1.0 / n, bc=(0, 0, 0, 0))
    d["dt"] = W.dt_from_cfl(ux, uy, T, d["dx"], 0.5, c_max=W.C_MAX_D1Q5)
    cfg = oracle.Config.from_dict(d)
    st = oracle.init(cfg, rho, ux, uy, T)
    out = oracle.run(cfg, st, 8)
    np.testing.assert_allclose(out.f, st.f, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(out.ux, st.ux, rtol=1e-13)
    np.testing.assert_allclose(out.T, st.T, rtol=1e-13)
