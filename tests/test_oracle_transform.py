"""Pins of the oracle's lattices, frame transformation and equilibria against
what the paper and the mathematics fix (no value here comes from the CUDA
path or from the oracle itself)."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden_table1():
    rows = []
    with open(os.path.join(HERE, "golden", "table1_lattices.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            model, node, weight = line.split()
            ev = lambda s: eval(s.replace("sqrt", "math.sqrt"), {"math": math})
            if node.startswith("+/-"):
                x = ev(node[3:])
                rows += [(model, -x, ev(weight)), (model, x, ev(weight))]
            else:
                rows.append((model, ev(node), ev(weight)))
    return rows


@pytest.mark.parametrize("q", [3, 4, 5])
def test_lattice_matches_table1_and_gauss_hermite(q):
    c, w, K = oracle.lattice(q)
    gold = sorted([(x, wt) for m, x, wt in _golden_table1() if m == "D1Q%d" % q])
    np.testing.assert_allclose(c, [x for x, _ in gold], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [wt for _, wt in gold], rtol=0, atol=1e-15)
    # the library's probabilists' Gauss-Hermite rule, normalised to unit mass
    xg, wg = He.hermegauss(q)
    np.testing.assert_allclose(c, xg, atol=1e-14)
    np.testing.assert_allclose(w, wg / math.sqrt(2 * math.pi), atol=1e-15)
    # moments of the unit Gaussian up to degree 2q-1: 1, 0, 1, 0, 3, 0, 15
    gauss = [1, 0, 1, 0, 3, 0, 15, 0, 105, 0]
    for k in range(2 * q):
        assert abs(np.sum(w * c**k) - gauss[k]) < 1e-12
    assert K == q - 1


def _vel(q, D, u, T):
    c, _, _ = oracle.lattice(q)
    u = np.atleast_1d(np.asarray(u, dtype=float))
    if D == 1:
        return (math.sqrt(T) * c + u[0])[:, None]
    cx = np.tile(c, q)
    cy = np.repeat(c, q)
    return np.stack([math.sqrt(T) * cx + u[0], math.sqrt(T) * cy + u[1]], axis=1)


def _moment_matrix(q, D, u, T, K=None):
    """Raw-moment matrix M(lambda): rows v_x^a v_y^b for a, b < q (Appendix B)."""
    v = _vel(q, D, u, T)
    rows = []
    for a in range(q):
        for b in range(q if D == 2 else 1):
            if K is not None and a + b > K:
                continue
            rows.append(v[:, 0] ** a * (v[:, 1] ** b if D == 2 else 1.0))
    return np.array(rows)


FRAMES = [((0.3, -0.2), 1.0, (0.1, 0.4), 1.3), ((2.4, 1.3), 0.7, (1.9, 1.0), 0.9),
          ((-1.0, 0.5), 2.0, (0.0, 0.0), 1.0), ((5.0, -3.0), 0.05, (4.8, -2.9), 0.06)]


@pytest.mark.parametrize("q,D", [(4, 1), (3, 1), (4, 2), (3, 2), (5, 1)])
@pytest.mark.parametrize("fr", range(len(FRAMES)))
def test_transform_equals_appendix_b_matrix_form(q, D, fr):
    """Tensor transformation == M(lambda')^-1 M(lambda) (Appendix B)."""
    u, T, up, Tp = FRAMES[fr]
    rng = np.random.default_rng(7 + fr)
    f = rng.uniform(0.1, 1.0, q**D)
    got = oracle.transform(q, D, f, u, T, up, Tp)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    Ms = _moment_matrix_mp(mp, q, D, u, T)
    Mt = _moment_matrix_mp(mp, q, D, up, Tp)
    rhs = Ms * mp.matrix([mp.mpf(float(x)) for x in f])
    want = np.array([float(x) for x in mp.lu_solve(Mt, rhs)])
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-12 * np.abs(f).sum())


def _moment_matrix_mp(mp, q, D, u, T):
    """M(lambda) of Appendix B in 50-digit arithmetic (the raw-moment
    Vandermonde system is ill conditioned for large |u|)."""
    c, _, _ = oracle.lattice(q)
    cm = [mp.mpf(float(x)) for x in c]
    sT = mp.sqrt(mp.mpf(T))
    u = list(np.atleast_1d(np.asarray(u, dtype=float))) + [0.0]
    if D == 1:
        v = [(sT * x + mp.mpf(u[0]), mp.mpf(0)) for x in cm]
    else:
        v = [(sT * cm[j % q] + mp.mpf(u[0]), sT * cm[j // q] + mp.mpf(u[1])) for j in range(q * q)]
    rows = [(a, b) for a in range(q) for b in range(q if D == 2 else 1)]
    M = mp.matrix(len(rows), len(v))
    for r, (a, b) in enumerate(rows):
        for j, (vx, vy) in enumerate(v):
            M[r, j] = vx**a * (vy**b if D == 2 else 1)
    return M


@pytest.mark.parametrize("q,D", [(4, 1), (4, 2), (3, 2)])
def test_transform_identity_and_round_trip(q, D):
    rng = np.random.default_rng(3)
    f = rng.uniform(0.1, 1.0, q**D)
    u, T = (0.7, -0.4), 1.3
    np.testing.assert_allclose(oracle.transform(q, D, f, u, T, u, T), f, rtol=0, atol=1e-14)
    g = oracle.transform(q, D, f, u, T, (1.5, 0.2), 0.6)
    back = oracle.transform(q, D, g, (1.5, 0.2), 0.6, u, T)
    np.testing.assert_allclose(back, f, rtol=0, atol=2e-13)


@pytest.mark.parametrize("grad_k", [0, 1])
def test_transform_keeps_moments_up_to_K(grad_k):
    """Moments of order <= K are frame invariant (Eq. eq:Mcondition)."""
    q, D = 4, 2
    rng = np.random.default_rng(11)
    f = rng.uniform(0.1, 1.0, q**D)
    u, T, up, Tp = (0.4, -1.1), 1.7, (-0.3, 0.2), 0.8
    g = oracle.transform(q, D, f, u, T, up, Tp, grad_k=grad_k)
    Ms = _moment_matrix(q, D, u, T, K=3)
    Mt = _moment_matrix(q, D, up, Tp, K=3)
    np.testing.assert_allclose(Mt @ g, Ms @ f, rtol=1e-12)


def test_grad_k_projection_has_no_coefficients_above_K():
    """Grad projection of order K (Eq. GradsProjection): f'/W is a polynomial of
    total degree <= 3 in c, i.e. its Hermite coefficients with a+b > 3 vanish."""
    q, D = 4, 2
    c, w, _ = oracle.lattice(q)
    rng = np.random.default_rng(5)
    f = rng.uniform(0.1, 1.0, q**D)
    g = oracle.transform(q, D, f, (0.2, 0.1), 1.0, (0.9, -0.5), 1.4, grad_k=1)
    cx, cy = np.tile(c, q), np.repeat(c, q)
    for a in range(4):
        for b in range(4):
            coef = np.sum(g * He.hermeval(cx, np.eye(5)[a]) * He.hermeval(cy, np.eye(5)[b]))
            if a + b > 3:
                assert abs(coef) < 1e-13
    # the tensor-product variant keeps them
    g2 = oracle.transform(q, D, f, (0.2, 0.1), 1.0, (0.9, -0.5), 1.4, grad_k=0)
    coef33 = np.sum(g2 * He.hermeval(cx, np.eye(5)[3]) * He.hermeval(cy, np.eye(5)[3]))
    assert abs(coef33) > 1e-3


def _raw_moments_1d(f, v):
    return [np.sum(f * v**k) for k in range(4)]


@pytest.mark.parametrize("fr", range(len(FRAMES)))
def test_expansion_coefficients_match_appendix_a_1d(fr):
    """alpha^(0..3) of Appendix A from the raw moments; alpha^(2) with the
    reading T delta + u u (the printed T delta - u u M0 fails, checked below)."""
    u, T, up, Tp = FRAMES[fr]
    q = 4
    c, w, _ = oracle.lattice(q)
    rng = np.random.default_rng(fr)
    f = rng.uniform(0.1, 1.0, q)
    M0, M1, M2, M3 = _raw_moments_1d(f, math.sqrt(T) * c + u[0])
    g = oracle.transform(q, 1, f, u, T, up, Tp)
    alpha = [np.sum(g * He.hermeval(c, np.eye(4)[n])) for n in range(4)]
    U, TT = up[0], Tp
    a0 = M0
    a1 = (M1 - U * M0) / math.sqrt(TT)
    a2 = (M2 - M0 * (TT + U * U) - 2 * U * (M1 - U * M0)) / TT
    a3 = (M3 - U**3 * M0 - 3 * (M1 - M0 * U) * (TT - U * U) - 3 * (M2 - M0 * U * U) * U) / TT**1.5
    np.testing.assert_allclose(alpha, [a0, a1, a2, a3], rtol=1e-11, atol=1e-11)
    a2_printed = (M2 - M0 * (TT - U * U * M0) - 2 * U * (M1 - U * M0)) / TT
    if abs(U) > 0.1:
        assert abs(a2_printed - alpha[2]) > 1e-3


def test_expansion_coefficients_match_appendix_a_2d_tensors():
    """Appendix A's tensor formulas for alpha^(1), alpha^(2), alpha^(3) in 2D
    against the coefficients of the oracle's transform."""
    q, D = 4, 2
    c, w, _ = oracle.lattice(q)
    rng = np.random.default_rng(21)
    f = rng.uniform(0.1, 1.0, q**D)
    u, T, up, Tp = (0.3, -0.6), 1.2, (1.1, 0.4), 0.7
    v = _vel(q, D, u, T)
    M0 = f.sum()
    M1 = np.einsum("i,ia->a", f, v)
    M2 = np.einsum("i,ia,ib->ab", f, v, v)
    M3 = np.einsum("i,ia,ib,ic->abc", f, v, v, v)
    U = np.asarray(up)
    I = np.eye(2)
    a1 = (M1 - U * M0) / math.sqrt(Tp)
    d1 = M1 - M0 * U
    a2 = (M2 - M0 * (Tp * I + np.outer(U, U)) - (np.outer(U, d1) + np.outer(d1, U))) / Tp
    t1 = np.einsum("a,bc->abc", d1, Tp * I - np.outer(U, U))
    cyc1 = t1 + np.transpose(t1, (1, 0, 2)) + np.transpose(t1, (1, 2, 0))
    d2 = M2 - M0 * np.outer(U, U)
    t2 = np.einsum("ab,c->abc", d2, U)
    cyc2 = t2 + np.transpose(t2, (0, 2, 1)) + np.transpose(t2, (2, 1, 0))
    a3 = (M3 - np.einsum("a,b,c->abc", U, U, U) * M0 - cyc1 - cyc2) / Tp**1.5
    g = oracle.transform(q, D, f, u, T, up, Tp)
    cx, cy = np.tile(c, q), np.repeat(c, q)
    h = lambda n, x: He.hermeval(x, np.eye(5)[n])
    A = lambda a, b: np.sum(g * h(a, cx) * h(b, cy))
    assert abs(A(0, 0) - M0) < 1e-12
    np.testing.assert_allclose([A(1, 0), A(0, 1)], a1, rtol=1e-11)
    np.testing.assert_allclose([A(2, 0), A(1, 1), A(0, 2)], [a2[0, 0], a2[0, 1], a2[1, 1]], rtol=1e-10,
                               atol=1e-11)
    np.testing.assert_allclose([A(3, 0), A(2, 1), A(1, 2), A(0, 3)],
                               [a3[0, 0, 0], a3[0, 0, 1], a3[0, 1, 1], a3[1, 1, 1]], rtol=1e-10, atol=1e-11)


def _mb_moments(rho, u, T, D):
    """Maxwell-Boltzmann moments J, P, Q, q, R of Sec. II.D."""
    u = np.asarray(u[:D], dtype=float)
    I = np.eye(D)
    J = rho * u
    P = rho * T * I + rho * np.outer(u, u)
    t = np.einsum("a,bc->abc", u, I)
    Q = rho * T * (t + np.transpose(t, (1, 0, 2)) + np.transpose(t, (1, 2, 0))) + rho * np.einsum(
        "a,b,c->abc", u, u, u)
    u2 = u @ u
    qv = rho * u * (u2 + T * (D + 2))
    R = rho * T * ((D + 2) * T + u2) * I + rho * ((D + 4) * T + u2) * np.outer(u, u)
    return J, P, Q, qv, R


def _lattice_moments(f, v):
    J = np.einsum("i,ia->a", f, v)
    P = np.einsum("i,ia,ib->ab", f, v, v)
    Q = np.einsum("i,ia,ib,ic->abc", f, v, v, v)
    v2 = np.einsum("ia,ia->i", v, v)
    qv = np.einsum("i,i,ia->a", f, v2, v)
    R = np.einsum("i,i,ia,ib->ab", f, v2, v, v)
    return J, P, Q, qv, R


@pytest.mark.parametrize("D", [1, 2])
def test_comoving_equilibrium_has_mb_moments(D):
    """rho W in the co-moving frame reproduces J, P, Q, q, R of Sec. II.D."""
    q = 4
    _, w, _ = oracle.lattice(q)
    W = w if D == 1 else np.outer(w, w).reshape(-1)
    rho, u, T = 1.3, (1.7, -0.8), 0.6
    v = _vel(q, D, u, T)
    got = _lattice_moments(rho * W, v)
    want = _mb_moments(rho, u, T, D)
    for g_, w_ in zip(got, want):
        np.testing.assert_allclose(g_, w_, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("grad_k", [0, 1])
def test_noncomoving_equilibrium_matches_mb_up_to_q_and_deviation_r(grad_k):
    """rho G W in a foreign frame: J, P, Q equal their MB values (Sec. II.D.1);
    the fourth moment deviates by R' (Eq. DeviationR)."""
    q, D = 4, 2
    rho, u, T = 0.9, np.array([1.2, -0.4]), 1.1
    ub, Tb = np.array([0.5, 0.3]), 0.8
    feq = oracle.equilibrium(q, D, rho, u, T, ub, Tb, grad_k=grad_k)
    v = _vel(q, D, ub, Tb)
    J, P, Q, qv, R = _lattice_moments(feq, v)
    Jm, Pm, Qm, qm, Rm = _mb_moments(rho, u, T, D)
    np.testing.assert_allclose(J, Jm, rtol=1e-12)
    np.testing.assert_allclose(P, Pm, rtol=1e-12)
    np.testing.assert_allclose(Q, Qm, rtol=1e-12, atol=1e-12)
    xi, th = u - ub, T - Tb
    I = np.eye(D)
    Rp = -rho * (np.outer(xi, xi) * (xi @ xi) + th * ((D + 2) * th * I + (xi @ xi) * I + (D + 4) * np.outer(xi, xi)))
    if grad_k:
        np.testing.assert_allclose(R - Rm, Rp, rtol=1e-10, atol=1e-12)
    # per axis (the 1D statement of Eq. DeviationR, D = 1) for the tensor product
    vx4 = np.sum(feq * v[:, 0] ** 4)
    mb4 = rho * (u[0] ** 4 + 6 * u[0] ** 2 * T + 3 * T**2)
    if not grad_k:
        assert abs((vx4 - mb4) - (-rho * (xi[0] ** 4 + 6 * th * xi[0] ** 2 + 3 * th**2))) < 1e-11


def test_deviation_r_1d():
    """Eq. DeviationR with D = 1 on D1Q4."""
    rho, u, T, ub, Tb = 1.4, 0.9, 1.3, -0.2, 0.7
    feq = oracle.equilibrium(4, 1, rho, [u], T, [ub], Tb)
    c, _, _ = oracle.lattice(4)
    v = math.sqrt(Tb) * c + ub
    xi, th = u - ub, T - Tb
    dev = np.sum(feq * v**4) - rho * (u**4 + 6 * u**2 * T + 3 * T**2)
    assert abs(dev - (-rho * (xi**4 + 6 * th * xi**2 + 3 * th**2))) < 1e-12


@pytest.mark.parametrize("q,D", [(4, 1), (3, 1), (4, 2), (3, 2)])
def test_equilibrium_equals_gaussian_expectation(q, D):
    """rho G W equals the Grad expansion whose coefficients are Gaussian
    expectations E[He_n((v - u')/sqrt(T'))], v ~ N(u, T) (Gauss-Hermite exact
    to degree 2q-1), computed here with a 30-point library quadrature."""
    rho, u, T, up, Tp = 1.1, np.array([0.8, -1.3]), 0.9, np.array([0.2, -0.7]), 1.4
    xg, wg = He.hermegauss(30)
    wg = wg / math.sqrt(2 * math.pi)
    c, w, K = oracle.lattice(q)

    def E(n, ax):
        z = (math.sqrt(T) * xg + u[ax] - up[ax]) / math.sqrt(Tp)
        return np.sum(wg * He.hermeval(z, np.eye(6)[n]))

    if D == 1:
        want = rho * w * sum(He.hermeval(c, np.eye(6)[n]) * E(n, 0) / math.factorial(n)
                             for n in range(K + 1))
    else:
        cx, cy = np.tile(c, q), np.repeat(c, q)
        W = np.outer(w, w).reshape(-1)
        want = rho * W * sum(He.hermeval(cx, np.eye(6)[a]) * He.hermeval(cy, np.eye(6)[b]) * E(a, 0) * E(b, 1)
                             / (math.factorial(a) * math.factorial(b))
                             for a in range(K + 1) for b in range(K + 1))
    got = oracle.equilibrium(q, D, rho, u[:D], T, up[:D], Tp)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)
