"""Seeded synthetic inputs: primitive initial fields and run settings.

This module holds no arithmetic of the PonD method itself: it only draws the
initial density, velocity and temperature fields (``numpy`` PCG64, seed
recorded) and fixes the run settings (relaxation time, time step, boundary
kinds).  Both the CUDA path and the CPU oracle start from what it returns.

Pressure enters only through the ideal-gas relation ``p = rho T`` of the
paper's equilibrium pressure tensor (Sec. II.D, P^MB = rho T I + rho u u).

Problems (sizes are the defaults; every generator takes smaller sizes for
tests):

* ``sod_1d``        1D Sod tube, 400 cells on [0, 1], zero-gradient ends,
                    BGK, tau = 1e-3, dt = 0.2/250 (250 steps to t = 0.2).
* ``pulse_2d``      2D periodic isobaric Gaussian pulse on [0,1)^2, 256^2,
                    background Mach 2 at 30 degrees, amplitude 0.1, seeded
                    centre and width in [0.05, 0.15], BGK, tau = 1e-4,
                    dt from CFL 0.2.
* ``riemann4_2d``   four-quadrant Riemann problem on [0,1]^2, 1024^2, seeded
                    quadrant states (rho in [0.1, 1.5], p in [0.03, 1.5],
                    Mach up to 3), zero-gradient, Pr = 0.71, minmod.
* ``config3_2d``    the paper's fixed Riemann configuration 3 (Sec. V.A.3).
* ``shock_bubble_2d`` planar Mach M shock into a Gaussian density bubble,
                    inflow on the left, zero-gradient elsewhere, Pr = 0.71.
* ``strong_shock_1d``, ``lax_1d``: the paper's 1D tubes (Sec. V.A.1, V.C.1).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4
# largest D1Q4 abscissa, sqrt(3 + sqrt(6)) (Table I); fixes dt from a CFL number
C_MAX_D1Q4 = math.sqrt(3.0 + math.sqrt(6.0))
# largest D1Q5 abscissa, sqrt(5 + sqrt(10)) (the D2Q25 f-lattice)
C_MAX_D1Q5 = math.sqrt(5.0 + math.sqrt(10.0))

BC_PERIODIC, BC_ZERO_GRADIENT, BC_INFLOW, BC_WALL = 0, 1, 2, 3
LIM_VANLEER, LIM_MINMOD = 0, 1


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def dt_from_cfl(ux, uy, T, dx, cfl, c_max=C_MAX_D1Q4):
    """dt such that max |v_{i alpha}| dt/dx = cfl on the initial state (Sec. V)."""
    ux = np.asarray(ux, dtype=np.float64)
    uy = np.asarray(uy, dtype=np.float64)
    vmax = np.max(np.maximum(np.abs(ux), np.abs(uy)) + np.sqrt(np.asarray(T)) * c_max)
    return float(cfl * dx / vmax)


def _base(D, nx, ny, **kw):
    d = dict(D=D, nx=nx, ny=ny if D == 2 else 1, qf=4, qg=3, gamma=GAMMA, tau=1e-4,
             prandtl=1.0, dx=1.0 / nx, dt=0.0, bc=(BC_ZERO_GRADIENT,) * 4,
             inflow=((0.0,) * 4,) * 4, grad_k=0, flux_appc=0, limiter=LIM_VANLEER,
             iterative=0, iter_tol=1e-12, iter_max=10)
    d.update(kw)
    return d


def sod_1d(n: int = 400, steps: int = 250, t_end: float = 0.2, cfl: float | None = None):
    """Sod tube: (rho, u, p) = (1, 0, 1) left of x = 0.5, (0.125, 0, 0.1) right."""
    x = (np.arange(n) + 0.5) / n
    left = x < 0.5
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    ux = np.zeros(n)
    T = p / rho
    cfg = _base(1, n, 1, tau=1e-3, dx=1.0 / n)
    if cfl is None:
        cfg["dt"] = t_end / steps
    else:
        cfg["dt"] = dt_from_cfl(ux, 0 * ux, T, 1.0 / n, cfl)
        steps = int(math.ceil(t_end / cfg["dt"]))
        cfg["dt"] = t_end / steps
    return dict(cfg=cfg, rho=rho, ux=ux, uy=np.zeros(n), T=T, steps=steps, t_end=t_end, x=x)


def tube_1d(n, left, right, x0=0.5, length=1.0, tau=1e-4, cfl=0.2, gamma=GAMMA, t_end=None):
    """Generic 1D Riemann tube from (rho, u, p) states on each side."""
    x = (np.arange(n) + 0.5) * (length / n)
    isl = x < x0
    rho = np.where(isl, left[0], right[0]).astype(np.float64)
    ux = np.where(isl, left[1], right[1]).astype(np.float64)
    p = np.where(isl, left[2], right[2]).astype(np.float64)
    T = p / rho
    dx = length / n
    cfg = _base(1, n, 1, tau=tau, dx=dx, gamma=gamma)
    cfg["dt"] = dt_from_cfl(ux, 0 * ux, T, dx, cfl)
    steps = None
    if t_end is not None:
        steps = int(math.ceil(t_end / cfg["dt"]))
        cfg["dt"] = t_end / steps
    return dict(cfg=cfg, rho=rho, ux=ux, uy=np.zeros(n), T=T, steps=steps, t_end=t_end, x=x)


def strong_shock_1d(n=800, cfl=0.2):
    """Strong shock tube (Sec. V.A.1): (1, 0, 1000) | (1, 0, 0.01), t = 0.012."""
    return tube_1d(n, (1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), tau=1e-6, cfl=cfl, t_end=0.012)


def lax_1d(n=600, cfl=0.2):
    """Lax tube (Sec. V.C.1): (0.445, 0.698, 3.528) | (0.5, 0, 0.571), t = 0.14."""
    return tube_1d(n, (0.445, 0.698, 3.528), (0.5, 0.0, 0.571), tau=1e-4, cfl=cfl, t_end=0.14)


def random_tube_1d(seed: int, n: int | None = None, steps: int | None = None):
    """Sod-type tube with seeded left/right states, rho in [0.1, 1.5], p in [0.03, 1.5]."""
    g = rng(seed)
    if n is None:
        n = int(round(math.exp(g.uniform(math.log(256), math.log(8192)))))
    rl, rr = g.uniform(0.1, 1.5, 2)
    pl, pr = g.uniform(0.03, 1.5, 2)
    w = tube_1d(n, (rl, 0.0, pl), (rr, 0.0, pr), tau=1e-4, cfl=0.2)
    w["steps"] = steps if steps is not None else int(g.integers(500, 5001))
    w["seed"] = seed
    return w


def pulse_2d(n: int = 256, seed: int = 0, steps: int = 1000, cfl: float = 0.2, mach: float = 2.0,
             angle_deg: float = 30.0, amp: float = 0.1, sigma: float | None = None,
             centre=None, tau: float = 1e-4):
    """Periodic isobaric Gaussian pulse advected at Mach ``mach`` (w.r.t. the
    background sound speed sqrt(gamma)) at ``angle_deg``; rho = 1 + amp g,
    T = 1/rho, g a periodic Gaussian with seeded centre and width (``sigma``
    and ``centre`` override the seeded values, for refinement studies at a
    fixed profile; the seeded draws are made either way)."""
    g = rng(seed)
    xc = g.uniform(0.0, 1.0, 2)
    sg = g.uniform(0.05, 0.15)
    sigma = sg if sigma is None else float(sigma)
    if centre is not None:
        xc = np.asarray(centre, dtype=np.float64)
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")  # [ny, nx]
    prof = np.zeros((n, n))
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            prof += np.exp(-((X - xc[0] - sx) ** 2 + (Y - xc[1] - sy) ** 2) / (2 * sigma**2))
    rho = 1.0 + amp * prof
    T = 1.0 / rho
    U = mach * math.sqrt(GAMMA)
    a = math.radians(angle_deg)
    ux = np.full((n, n), U * math.cos(a))
    uy = np.full((n, n), U * math.sin(a))
    cfg = _base(2, n, n, tau=tau, dx=1.0 / n, bc=(BC_PERIODIC,) * 4)
    cfg["dt"] = dt_from_cfl(ux, uy, T, 1.0 / n, cfl)
    return dict(cfg=cfg, rho=rho, ux=ux, uy=uy, T=T, steps=steps, seed=seed,
                centre=xc, sigma=sigma, amp=amp, velocity=(U * math.cos(a), U * math.sin(a)))


def pulse_exact_2d(w, t):
    """The pulse's initial density translated by u t (periodic): the exact
    Euler solution of an entropy wave (uniform pressure and velocity)."""
    n = w["cfg"]["nx"]
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    cx = (w["centre"][0] + w["velocity"][0] * t) % 1.0
    cy = (w["centre"][1] + w["velocity"][1] * t) % 1.0
    prof = np.zeros((n, n))
    for sx in (-1, 0, 1):
        for sy in (-1, 0, 1):
            prof += np.exp(-((X - cx - sx) ** 2 + (Y - cy - sy) ** 2) / (2 * w["sigma"] ** 2))
    return 1.0 + w["amp"] * prof


def _quadrants(n, states):
    """states: [(rho, ux, uy, p)] for quadrants NE, NW, SW, SE (split at 0.5)."""
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    rho = np.empty((n, n)); ux = np.empty((n, n)); uy = np.empty((n, n)); p = np.empty((n, n))
    masks = [(X > 0.5) & (Y > 0.5), (X <= 0.5) & (Y > 0.5), (X <= 0.5) & (Y <= 0.5),
             (X > 0.5) & (Y <= 0.5)]
    for m, s in zip(masks, states):
        rho[m], ux[m], uy[m], p[m] = s
    return rho, ux, uy, p / rho


def riemann4_2d(n: int = 1024, seed: int = 0, steps: int = 200, cfl: float = 0.2,
                prandtl: float = 0.71):
    """Four-quadrant Riemann problem with seeded states: rho ~ U[0.1, 1.5],
    p ~ U[0.03, 1.5], Mach ~ U[0, 3] w.r.t. the local sound speed, direction
    ~ U[0, 2 pi)."""
    g = rng(seed)
    states = []
    for _ in range(4):
        r = g.uniform(0.1, 1.5)
        p = g.uniform(0.03, 1.5)
        M = g.uniform(0.0, 3.0)
        th = g.uniform(0.0, 2 * math.pi)
        cs = math.sqrt(GAMMA * p / r)
        states.append((r, M * cs * math.cos(th), M * cs * math.sin(th), p))
    rho, ux, uy, T = _quadrants(n, states)
    cfg = _base(2, n, n, tau=1e-4, dx=1.0 / n, prandtl=prandtl, limiter=LIM_MINMOD)
    cfg["dt"] = dt_from_cfl(ux, uy, T, 1.0 / n, cfl)
    return dict(cfg=cfg, rho=rho, ux=ux, uy=uy, T=T, steps=steps, seed=seed, states=states)


def config3_2d(n: int = 500, cfl: float = 0.2, prandtl: float = 1.0):
    """The paper's Riemann configuration 3 (Sec. V.A.3), zero-gradient ends."""
    states = [(1.5, 0.0, 0.0, 1.5), (0.5323, 1.206, 0.0, 0.3), (0.138, 1.206, 1.206, 0.029),
              (0.5323, 0.0, 1.206, 0.3)]
    rho, ux, uy, T = _quadrants(n, states)
    cfg = _base(2, n, n, tau=1e-4, dx=1.0 / n, prandtl=prandtl, limiter=LIM_MINMOD)
    cfg["dt"] = dt_from_cfl(ux, uy, T, 1.0 / n, cfl)
    return dict(cfg=cfg, rho=rho, ux=ux, uy=uy, T=T, steps=None, states=states)


def post_shock(M, rho1=1.0, p1=1.0, gamma=GAMMA):
    """Rankine-Hugoniot state behind a shock moving at Mach M into gas at rest."""
    c1 = math.sqrt(gamma * p1 / rho1)
    rho2 = rho1 * (gamma + 1) * M * M / ((gamma - 1) * M * M + 2)
    p2 = p1 * (2 * gamma * M * M - (gamma - 1)) / (gamma + 1)
    u2 = 2 * c1 / (gamma + 1) * (M - 1.0 / M)
    return rho2, u2, p2


def shock_bubble_2d(seed: int, n: int | None = None, steps: int = 500, cfl: float = 0.2,
                    prandtl: float = 0.71, side_range=(64, 512), tau: float = 1e-3):
    """Mach M in [1.5, 5] planar shock at x = 0.1 moving +x into (rho, p) = (1, 1)
    containing an isobaric Gaussian bubble at (0.4, 0.5), sigma 0.08, peak
    density ratio r ~ log-U[0.1, 10]; inflow at the post-shock state on the
    left, zero-gradient elsewhere.  tau = 1e-3 (mu = tau rho T ~ 1e-3, the
    viscosity range of Sec. V): with 1e-4 the smallest grids run at
    dt/tau ~ 3-7, where the explicit quasi-equilibrium half steps amplify
    third-order modes faster than the BGK factor damps them."""
    g = rng(seed)
    if n is None:
        n = int(round(math.exp(g.uniform(math.log(side_range[0]), math.log(side_range[1])))))
    M = g.uniform(1.5, 5.0)
    ratio = math.exp(g.uniform(math.log(0.1), math.log(10.0)))
    x = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(x, x, indexing="xy")
    bub = np.exp(-((X - 0.4) ** 2 + (Y - 0.5) ** 2) / (2 * 0.08**2))
    rho = 1.0 + (ratio - 1.0) * bub
    p = np.ones((n, n))
    ux = np.zeros((n, n))
    uy = np.zeros((n, n))
    r2, u2, p2 = post_shock(M)
    behind = X < 0.1
    rho[behind], ux[behind], p[behind] = r2, u2, p2
    T = p / rho
    inflow = ((r2, u2, 0.0, p2 / r2), (0.0,) * 4, (0.0,) * 4, (0.0,) * 4)
    cfg = _base(2, n, n, tau=tau, dx=1.0 / n, prandtl=prandtl, limiter=LIM_MINMOD,
                bc=(BC_INFLOW, BC_ZERO_GRADIENT, BC_ZERO_GRADIENT, BC_ZERO_GRADIENT),
                inflow=inflow)
    cfg["dt"] = dt_from_cfl(ux, uy, T, 1.0 / n, cfl)
    return dict(cfg=cfg, rho=rho, ux=ux, uy=uy, T=T, steps=steps, seed=seed, mach=M, ratio=ratio)


def thermal_couette_2d(ny: int = 16, nx: int = 8, prandtl: float = 1.0, ec: float = 20.0,
                      mach: float = 0.5, re: float = 20.0, t_cold: float = 1.0, cfl: float = 0.2,
                      gamma: float = GAMMA):
    """Thermal Couette flow (Sec. V.B.2): walls on the y sides, the lower one at
    rest at T_C, the upper one moving at u0 = Ma sqrt(gamma T_C) at
    T_H = T_C + u0^2 / (C_p Ec); periodic in x; Re = rho u0 L / mu with L = 1
    (ny cells), mu = tau rho T.  Starts from the analytic steady state
    ``theta(y)`` = (T - T_C)/(T_H - T_C) = y + Pr Ec/2 y (1 - y) with the linear
    velocity and uniform pressure 1."""
    cp = gamma / (gamma - 1.0)
    u0 = mach * math.sqrt(gamma * t_cold)
    dT = u0 * u0 / (cp * ec)
    y = (np.arange(ny) + 0.5) / ny

    def theta(yy):
        return yy + 0.5 * prandtl * ec * yy * (1.0 - yy)

    T = np.repeat((t_cold + dT * theta(y))[:, None], nx, axis=1)
    rho = 1.0 / T
    ux = np.repeat((u0 * y)[:, None], nx, axis=1)
    uy = np.zeros((ny, nx))
    tau = u0 / re  # mu = rho u0 L / Re, and rho T = 1
    inflow = ((0.0,) * 4, (0.0,) * 4, (0.0, 0.0, 0.0, t_cold), (0.0, u0, 0.0, t_cold + dT))
    cfg = _base(2, nx, ny, tau=tau, dx=1.0 / ny, prandtl=prandtl, gamma=gamma,
                bc=(BC_PERIODIC, BC_PERIODIC, BC_WALL, BC_WALL), inflow=inflow)
    cfg["dt"] = dt_from_cfl(ux, uy, T, 1.0 / ny, cfl)
    return dict(cfg=cfg, rho=rho, ux=ux, uy=uy, T=T, y=y, u0=u0, t_cold=t_cold, dT=dT,
                theta=theta)


def random_state_grid(D: int, nx: int, ny: int, seed: int, mach: float = 1.0, rho=(0.5, 1.5),
                      T=(0.5, 2.0)):
    """Smooth-ish random primitive fields for parity tests on tiny grids."""
    g = rng(seed)
    shp = (ny if D == 2 else 1, nx)
    r = g.uniform(*rho, shp)
    t = g.uniform(*T, shp)
    cs = np.sqrt(GAMMA * t)
    ux = mach * cs * g.uniform(-1, 1, shp)
    uy = mach * cs * g.uniform(-1, 1, shp) if D == 2 else np.zeros(shp)
    return r, ux, uy, t
