"""Pins of the oracle's quasi-equilibrium relaxation and macroscopic moments
(Sec. III.A, Eq. eq::quasi_f; Sec. IV.B, Eq. QE_relaxation)."""
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He

import oracle

GAMMA = 1.4
CV = 1.0 / (GAMMA - 1.0)


def _cells(D, seed):
    """A non-equilibrium cell in its co-moving frame: populations of a random
    state moved into the frame of their own (u, T)."""
    rng = np.random.default_rng(seed)
    f0 = rng.uniform(0.2, 1.0, 4**D)
    g0 = rng.uniform(0.2, 1.0, 3**D)
    u0, T0 = rng.uniform(-1, 1, 2), rng.uniform(0.5, 1.5)
    m, ok = oracle.macro(4, 3, D, GAMMA, f0, g0, u0[:D], T0)
    assert ok
    rho, ux, uy, T = m
    u = np.array([ux, uy])
    f = oracle.transform(4, D, f0, u0[:D], T0, u[:D], T)
    g = oracle.transform(3, D, g0, u0[:D], T0, u[:D], T)
    return f, g, u, T, rho


def _conserved(D, f, g, u, T):
    m, _ = oracle.macro(4, 3, D, GAMMA, f, g, u[:D], T)
    rho, ux, uy, TT = m
    return np.array([rho, rho * ux, rho * uy, CV * rho * TT + 0.5 * rho * (ux * ux + uy * uy)])


@pytest.mark.parametrize("D", [1, 2])
def test_macro_matches_conservation_laws(D):
    """rho, rho u, rho E of Eq. eq::ConservationLaws with E of Eq. eq:E,
    recomputed here from the raw sums."""
    rng = np.random.default_rng(1)
    f, g = rng.uniform(0.1, 1, 4**D), rng.uniform(0.1, 1, 3**D)
    uf, Tf = rng.uniform(-1, 1, 2), 0.8
    c4, _, _ = oracle.lattice(4)
    if D == 1:
        vx, vy = math.sqrt(Tf) * c4 + uf[0], 0 * c4
    else:
        vx, vy = math.sqrt(Tf) * np.tile(c4, 4) + uf[0], math.sqrt(Tf) * np.repeat(c4, 4) + uf[1]
    rho = f.sum()
    jx, jy = (vx * f).sum(), (vy * f).sum()
    rhoE = (0.5 * (vx**2 + vy**2) * f).sum() + g.sum()
    m, ok = oracle.macro(4, 3, D, GAMMA, f, g, uf[:D], Tf)
    assert ok
    assert abs(m[0] - rho) < 1e-14
    assert abs(m[1] - jx / rho) < 1e-13
    if D == 2:
        assert abs(m[2] - jy / rho) < 1e-13
    T = (rhoE - 0.5 * (jx**2 + jy**2) / rho) / (CV * rho)
    assert abs(m[3] - T) < 1e-13


@pytest.mark.parametrize("D", [1, 2])
def test_qe_identity_when_pr_is_one(D):
    f, g, u, T, _ = _cells(D, 3)
    f2, g2 = oracle.qe_half(4, 3, D, GAMMA, 0.01, 1e-2, 1e-2, f, g, u[:D], T)
    np.testing.assert_array_equal(f2, f)
    np.testing.assert_array_equal(g2, g)


@pytest.mark.parametrize("D", [1, 2])
def test_qe_conserves_mass_momentum_energy(D):
    f, g, u, T, _ = _cells(D, 4)
    f2, g2 = oracle.qe_half(4, 3, D, GAMMA, 0.01, 1e-2, 1e-2 / 0.71, f, g, u[:D], T)
    np.testing.assert_allclose(_conserved(D, f2, g2, u, T), _conserved(D, f, g, u, T), rtol=1e-13,
                               atol=1e-14)
    assert np.max(np.abs(f2 - f)) > 1e-6


@pytest.mark.parametrize("D", [1, 2])
def test_qe_state_keeps_heat_flux_tensor(D):
    """f* of Eq. eq::quasi_f has the same third-order non-equilibrium flux Q as f,
    and g* the same varsigma (by Hermite orthogonality)."""
    f, g, u, T, rho = _cells(D, 5)
    dt, t1, t2 = 0.01, 1e-2, 1e-2 / 0.5
    k = 0.5 * dt * (1 / t1 - 1 / t2)
    f2, g2 = oracle.qe_half(4, 3, D, GAMMA, dt, t1, t2, f, g, u[:D], T)
    c4, w4, _ = oracle.lattice(4)
    c3, w3, _ = oracle.lattice(3)
    if D == 1:
        e4, W4 = (math.sqrt(T) * c4)[:, None], w4
        e3, W3 = (math.sqrt(T) * c3)[:, None], w3
    else:
        e4 = math.sqrt(T) * np.stack([np.tile(c4, 4), np.repeat(c4, 4)], 1)
        e3 = math.sqrt(T) * np.stack([np.tile(c3, 3), np.repeat(c3, 3)], 1)
        W4, W3 = np.outer(w4, w4).reshape(-1), np.outer(w3, w3).reshape(-1)
    feq = rho * W4
    geq = (CV - 0.5 * D) * T * rho * W3
    fstar = feq + (f2 - f) / k
    gstar = geq + (g2 - g) / k
    Q = lambda h: np.einsum("i,ia,ib,ic->abc", h, e4, e4, e4)
    np.testing.assert_allclose(Q(fstar - feq), Q(f - feq), rtol=1e-11, atol=1e-12)
    vs = lambda h: np.einsum("i,ia->a", h, e3)
    np.testing.assert_allclose(vs(gstar - geq), vs(g - geq), rtol=1e-11, atol=1e-12)


def test_qe_change_is_third_order_hermite_content():
    """In the co-moving frame f* - f^eq is the total-order-3 part of the Hermite
    expansion of f - f^eq (library Hermite polynomials), and g* - g^eq the
    first-order part of g - g^eq."""
    D = 2
    f, g, u, T, rho = _cells(D, 6)
    dt, t1, t2 = 0.02, 1e-2, 1e-2 / 0.71
    k = 0.5 * dt * (1 / t1 - 1 / t2)
    f2, g2 = oracle.qe_half(4, 3, D, GAMMA, dt, t1, t2, f, g, u, T)
    c4, w4, _ = oracle.lattice(4)
    cx, cy = np.tile(c4, 4), np.repeat(c4, 4)
    W = np.outer(w4, w4).reshape(-1)
    h = lambda n, x: He.hermeval(x, np.eye(5)[n])
    fneq = f - rho * W
    want = np.zeros(16)
    for a in range(4):
        for b in range(4):
            if a + b == 3:
                A = np.sum(fneq * h(a, cx) * h(b, cy))
                want += W * A * h(a, cx) * h(b, cy) / (math.factorial(a) * math.factorial(b))
    np.testing.assert_allclose((f2 - f) / k, want, rtol=1e-10, atol=1e-12)
    c3, w3, _ = oracle.lattice(3)
    gx, gy = np.tile(c3, 3), np.repeat(c3, 3)
    W3 = np.outer(w3, w3).reshape(-1)
    gneq = g - (CV - 1.0) * T * rho * W3
    wantg = W3 * (np.sum(gneq * gx) * gx + np.sum(gneq * gy) * gy)
    np.testing.assert_allclose((g2 - g) / k, wantg, rtol=1e-10, atol=1e-12)
