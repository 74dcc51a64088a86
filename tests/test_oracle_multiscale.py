"""Multiscale f-lattice of the oracle (Sec. II.E lifting and projection,
Sec. IV.C switching, Sec. V.C.1 Lax tube): each step every cell takes D1Q4 /
D2Q16 where a velocity or temperature jump across it exceeds a threshold and
D1Q3 / D2Q9 elsewhere; a face takes the higher lattice of its two cells.
Pins:

* lifting equals the Grad expansion's continuous Hermite moments in the new
  frame (40-node Gauss-Hermite quadrature of the expansion, a
  different computation), and projection keeps every moment of order <= 2 per
  axis;
* same-frame lifting and projection are inverse to rounding;
* all cells high is the plain D2Q16 step bit for bit, all cells low the plain
  D2Q9 f-lattice step to rounding;
* the switching measure in closed form on step profiles, with its boundary
  rules;
* conservation with mixed lattices: mass and momentum in the main flux form,
  and energy as well in Appendix C's form (the low lattice does not carry the
  third-order moment the energy flux needs in another frame);
* the Lax tube against its exact solution: D1Q3 alone does not converge (an
  error at the Euler level, the paper's observation), D1Q4 does, and the
  multiscale run matches D1Q4 with a few percent of cells on the high lattice.
"""
import math

import numpy as np
import pytest

import oracle
from tests import riemann_exact as RE
from paper_2302_00310_gb300 import workloads as W

GAMMA = 1.4


def _he(n, x):
    return [np.ones_like(x), x, x * x - 1, x**3 - 3 * x][n]


def _lattice_moments(q, D, f, u, T, a_max):
    c, _, _ = oracle.lattice(q)
    sT = math.sqrt(T)
    if D == 1:
        v = sT * c + u[0]
        return np.array([np.sum(f * v**a) for a in range(a_max + 1)])
    vx = sT * np.tile(c, q) + u[0]
    vy = sT * np.repeat(c, q) + u[1]
    return np.array([[np.sum(f * vx**a * vy**b) for b in range(a_max + 1)] for a in range(a_max + 1)])


@pytest.mark.parametrize("D", [1, 2])
def test_lifting_is_the_grad_expansion_moved(D):
    """D1Q3 populations in {u, T} lifted onto D1Q4 in {u', T'}: the
    coefficients are the Hermite moments, in the new frame, of the continuous
    Grad expansion sum_n alpha_n He_n / n! times the Gaussian of {u, T}."""
    g = np.random.default_rng(3 + D)
    q3 = 3**D
    f3 = g.uniform(0.1, 1.0, q3)
    u, T, up, Tp = (0.4, -0.3), 0.8, (-0.2, 0.5), 1.3
    got = oracle.transform_x(3, 4, 3, D, f3, u, T, up, Tp)
    c3, _, _ = oracle.lattice(3)
    c4, w4, _ = oracle.lattice(4)
    # the source's own coefficients, alpha_ab = sum_j f_j He_a(c_xj) He_b(c_yj)
    if D == 1:
        alpha = np.array([np.sum(f3 * _he(a, c3)) for a in range(3)])
    else:
        cx, cy = np.tile(c3, 3), np.repeat(c3, 3)
        alpha = np.array([[np.sum(f3 * _he(a, cx) * _he(b, cy)) for b in range(3)] for a in range(3)])
    z, wz = np.polynomial.hermite_e.hermegauss(40)
    wz = wz / math.sqrt(2 * math.pi)
    sT, sTp = math.sqrt(T), math.sqrt(Tp)

    def proj(d, n):  # E[He_n((u_d + sT Z - up_d)/sTp) He_k(Z)] / k!, k = 0..2
        xi = (u[d] + sT * z - up[d]) / sTp
        return np.array([np.sum(wz * _he(n, xi) * _he(k, z)) / math.factorial(k) for k in range(3)])

    if D == 1:
        ap = np.array([proj(0, n) @ alpha for n in range(4)])
        want = w4 * sum(ap[n] * _he(n, c4) / math.factorial(n) for n in range(4))
    else:
        ap = np.array([[proj(0, a) @ alpha @ proj(1, b) for b in range(4)] for a in range(4)])
        cx, cy = np.tile(c4, 4), np.repeat(c4, 4)
        W4 = np.outer(w4, w4).ravel()
        want = W4 * sum(ap[a, b] * _he(a, cx) * _he(b, cy) / (math.factorial(a) * math.factorial(b))
                        for a in range(4) for b in range(4))
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("D", [1, 2])
def test_projection_keeps_the_moments_of_order_two(D):
    g = np.random.default_rng(9 + D)
    f4 = g.uniform(0.1, 1.0, 4**D)
    u, T, up, Tp = (0.7, 0.2), 1.1, (0.1, -0.4), 0.6
    f3 = oracle.transform_x(4, 3, 2, D, f4, u, T, up, Tp)
    np.testing.assert_allclose(_lattice_moments(3, D, f3, up, Tp, 2),
                               _lattice_moments(4, D, f4, u, T, 2), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("grad_k", [0, 1])
def test_same_frame_lifting_and_projection_are_inverse(grad_k):
    g = np.random.default_rng(21)
    f3 = g.uniform(0.1, 1.0, 9)
    u, T = (0.3, -0.6), 0.9
    if grad_k:  # keep the source inside the Grad subspace a + b <= 2
        f3 = oracle.transform_x(3, 3, 2, 2, f3, u, T, u, T, grad_k=1)
    f4 = oracle.transform_x(3, 4, 2, 2, f3, u, T, u, T, grad_k=grad_k)
    back = oracle.transform_x(4, 3, 2, 2, f4, u, T, u, T, grad_k=grad_k)
    np.testing.assert_allclose(back, f3, rtol=1e-13, atol=1e-15)
    # the projection of a high-lattice state onto its own nodes is idempotent
    h = g.uniform(0.1, 1.0, 16)
    p1 = oracle.transform_x(4, 4, 2, 2, h, u, T, u, T, grad_k=grad_k)
    p2 = oracle.transform_x(4, 4, 2, 2, p1, u, T, u, T, grad_k=grad_k)
    np.testing.assert_allclose(p2, p1, rtol=1e-13, atol=1e-15)


def _case(D, n, seed, **kw):
    rho, ux, uy, T = W.random_state_grid(D, n, n, seed=seed, mach=0.8)
    d = W._base(D, n, n, **dict(dict(tau=5e-3, dx=1.0 / n), **kw))
    d["dt"] = W.dt_from_cfl(ux, uy, T, d["dx"], 0.3)
    return d, (rho, ux, uy, T)


WALLS_2D = ((0.0,) * 4, (0.0,) * 4, (0.0, 0.2, 0.0, 1.0), (0.0, -0.1, 0.0, 1.1))
WALLS_1D = ((0.0, 0.0, 0.0, 1.0), (0.0, 0.0, 0.0, 1.1), (0.0,) * 4, (0.0,) * 4)


@pytest.mark.parametrize("D,grad_k,appc,bc,pr", [(1, 0, 0, (1, 1, 0, 0), 1.0), (1, 0, 1, (0, 0, 0, 0), 1.0),
                                                 (2, 0, 0, (1, 1, 0, 0), 1.0), (2, 1, 1, (0, 0, 1, 2), 1.0),
                                                 (2, 0, 0, (0, 0, 0, 0), 0.71), (1, 0, 1, (1, 1, 0, 0), 0.5),
                                                 (2, 0, 0, (1, 1, 3, 3), 1.0), (2, 1, 1, (0, 0, 3, 3), 0.71),
                                                 (1, 0, 0, (3, 3, 0, 0), 0.71)])
def test_all_high_and_all_low_are_the_single_lattice_steps(D, grad_k, appc, bc, pr):
    """With the quasi-equilibrium step (Pr != 1) and walls too: a multiscale run
    whose cells are all high is the D2Q16 (D1Q4) run bit for bit, one whose
    cells are all low is the D2Q9 (D1Q3) f-lattice run to rounding (the QE
    step on a low cell relaxes the third-order content D2Q9 resolves; a low
    wall ghost carries the Chapman-Enskog content D2Q9 resolves)."""
    walls = 3 in bc
    d, fields = _case(D, 10, 40 + D, grad_k=grad_k, flux_appc=appc, bc=bc, prandtl=pr,
                      inflow=(WALLS_2D if D == 2 else WALLS_1D) if walls else ((1.1, 0.3, -0.1, 0.9),) * 4)
    steps = 3
    plain = oracle.Config.from_dict(d)
    high = oracle.Config.from_dict(dict(d, ms=1, ms_theta_u=-1.0, ms_theta_T=-1.0))
    a = oracle.run(plain, oracle.init(plain, *fields), steps)
    b = oracle.run(high, oracle.init(high, *fields), steps)
    assert np.array_equal(a.f, b.f) and np.array_equal(a.g, b.g) and np.array_equal(a.T, b.T)
    assert b.report["ms_high"] == steps * d["nx"] * d["ny"]
    q3 = oracle.Config.from_dict(dict(d, qf=3))
    low = oracle.Config.from_dict(dict(d, ms=1, ms_theta_u=1e30, ms_theta_T=1e30))
    a = oracle.run(q3, oracle.init(q3, *fields), steps)
    b = oracle.run(low, oracle.init(low, *fields), steps)
    assert b.report["ms_high"] == 0
    np.testing.assert_allclose(oracle.moments(low, b), oracle.moments(q3, a), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(b.g, a.g, rtol=1e-12, atol=1e-14)
    # the low cells' storage is the lifting of the D2Q9 populations
    for k in range(d["ny"]):
        for j in range(d["nx"]):
            u = (b.ux[k, j], b.uy[k, j])
            lifted = oracle.transform_x(3, 4, 2, D, a.f[:, k, j], u, b.T[k, j], u, b.T[k, j])
            np.testing.assert_allclose(b.f[:, k, j], lifted, rtol=1e-12, atol=1e-14)


def test_switching_measure_on_step_profiles():
    n = 8
    T = np.where(np.arange(n) < 5, 2.0, 0.5)[None, :].repeat(n, 0)
    ux = np.full((n, n), 0.3)
    uy = np.where(np.arange(n) < 3, 0.0, 0.6)[:, None].repeat(n, 1)
    for bc, wrap in (((1, 1, 1, 1), False), ((0, 0, 0, 0), True)):
        cfg = oracle.Config(D=2, nx=n, ny=n, bc=bc, ms=1)
        su, sT = oracle.ms_measure(cfg, ux, uy, T)
        want_T = np.zeros((n, n))
        want_T[:, 4] = 1.5 / (2 * 2.0)
        want_T[:, 5] = 1.5 / (2 * 0.5)
        want_u = np.zeros((n, n))
        want_u[2, :] = 0.6 / (2 * np.sqrt(T[2, :]))
        want_u[3, :] = 0.6 / (2 * np.sqrt(T[3, :]))
        if wrap:  # the jumps back at the periodic edges
            want_T[:, 0] = 1.5 / (2 * 2.0)
            want_T[:, n - 1] = 1.5 / (2 * 0.5)
            want_u[0, :] = 0.6 / (2 * np.sqrt(T[0, :]))
            want_u[n - 1, :] = 0.6 / (2 * np.sqrt(T[n - 1, :]))
        np.testing.assert_allclose(sT, want_T, rtol=1e-15, atol=0)
        np.testing.assert_allclose(su, want_u, rtol=1e-15, atol=0)


@pytest.mark.parametrize("D,appc,pr", [(1, 0, 1.0), (1, 1, 1.0), (2, 0, 1.0), (2, 1, 1.0), (2, 1, 0.71),
                                       (1, 0, 0.5)])
def test_conservation_with_mixed_lattices(D, appc, pr):
    n = 10
    d, fields = _case(D, n, 17, tau=2e-2, bc=(0, 0, 0, 0), flux_appc=appc, prandtl=pr)
    probe = oracle.Config.from_dict(dict(d, ms=1))
    su, sT = oracle.ms_measure(probe, *fields[1:])
    th = float(np.median(np.maximum(su, sT)))
    cfg = oracle.Config.from_dict(dict(d, ms=1, ms_theta_u=th, ms_theta_T=th))
    st = oracle.init(cfg, *fields)

    def totals(s):
        r, vx, vy, t = oracle.moments(cfg, s)
        return np.array([r.sum(), (r * vx).sum(), (r * vy).sum(),
                         (r * t / (GAMMA - 1) + 0.5 * r * (vx**2 + vy**2)).sum()])

    t0 = totals(st)
    out = oracle.run(cfg, st, 10)
    cells = 10 * n ** D
    assert 0.05 * cells < out.report["ms_high"] < 0.95 * cells
    rel = np.abs(totals(out) - t0) / np.array([t0[0], t0[0], t0[0], t0[3]])
    assert np.max(rel[:3]) < 1e-13
    if appc:
        assert rel[3] < 1e-13
    else:
        assert rel[3] > 1e-6  # the main form on the low lattice does not keep energy


def test_lax_tube_multiscale_matches_the_high_lattice():
    left, right = (0.445, 0.698, 3.528), (0.5, 0.0, 0.571)
    err, frac = {}, {}
    for n in (200, 400):
        w = W.lax_1d(n=n)
        exact = RE.solution(left, right, w["x"], w["t_end"])[0]
        for name, extra in (("q4", {}), ("q3", dict(qf=3)),
                            ("ms", dict(ms=1, ms_theta_u=0.05, ms_theta_T=0.05))):
            cfg = oracle.Config.from_dict(dict(w["cfg"], **extra))
            st = oracle.run(cfg, oracle.init(cfg, w["rho"], w["ux"], w["uy"], w["T"]), w["steps"])
            assert st.report["flags"] == 0
            err[name, n] = float(np.mean(np.abs(oracle.moments(cfg, st)[0][0] - exact)))
            frac[name, n] = st.report["ms_high"] / (w["steps"] * n)
    assert err["q3", 400] > 0.9 * err["q3", 200]          # D1Q3: no convergence
    assert err["q4", 400] < 0.8 * err["q4", 200]          # D1Q4 converges
    assert err["q3", 400] > 1.5 * err["q4", 400]
    for n in (200, 400):
        assert err["ms", n] < 1.02 * err["q4", n]
        assert 0.0 < frac["ms", n] < 0.1


def test_walled_channel_with_mixed_lattices_stays_mirror_symmetric():
    """A channel state mirror-symmetric about its mid-plane between two equal
    walls, with the QE step and thresholds that put part of the cells on each
    lattice: the lattice choice, the wall ghosts' lattices and the state stay
    symmetric."""
    nx, ny = 6, 12
    g = W.rng(5)
    half = [g.uniform(a, b, (ny // 2, nx)) for a, b in ((0.8, 1.2), (0.8, 1.2), (-0.3, 0.3), (-0.3, 0.3))]
    rho, T, ux = (np.vstack([a, a[::-1]]) for a in half[:3])
    uy = np.vstack([half[3], -half[3][::-1]])
    wall = (0.0, 0.1, 0.0, 1.05)
    d = W._base(2, nx, ny, tau=5e-3, dx=1.0 / ny, prandtl=0.71, bc=(0, 0, 3, 3), inflow=(wall,) * 4)
    d["dt"] = W.dt_from_cfl(ux, uy, T, d["dx"], 0.3)
    probe = oracle.Config.from_dict(dict(d, ms=1))
    su, sT = oracle.ms_measure(probe, ux, uy, T)
    th = float(np.median(np.maximum(su, sT)))
    cfg = oracle.Config.from_dict(dict(d, ms=1, ms_theta_u=th, ms_theta_T=th))
    st = oracle.run(cfg, oracle.init(cfg, rho, ux, uy, T), 6)
    assert 0 < st.report["ms_high"] < 6 * nx * ny
    m = oracle.moments(cfg, st)
    for field, sign in zip(m, (1, 1, -1, 1)):
        np.testing.assert_allclose(field, sign * field[::-1], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("bad", [dict(iterative=1), dict(qf=5)])
def test_multiscale_rejects_what_it_does_not_cover(bad):
    d, fields = _case(2, 8, 3)
    cfg = oracle.Config.from_dict(dict(d, ms=1, **bad))
    with pytest.raises(ValueError):
        oracle.init(cfg, *fields)
