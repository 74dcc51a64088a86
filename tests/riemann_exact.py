"""Exact solution of the 1D Riemann problem for the Euler equations of an
ideal gas, written from the textbook mathematics (wave curves through the
star region, Newton iteration on the star pressure, self-similar sampling).
Used only as an independent reference for the Sod-type tests.
"""
from __future__ import annotations

import math

import numpy as np


def _wave(p, rho, pk, ck, gamma):
    """Velocity jump across the left/right wave as a function of the star
    pressure p (shock if p > pk, rarefaction otherwise), and its derivative."""
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    e = (gamma - 1.0) / (2.0 * gamma)
    return (2.0 * ck / (gamma - 1.0)) * ((p / pk) ** e - 1.0), (1.0 / (rho * ck)) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))


def star_state(left, right, gamma=1.4, tol=1e-14):
    """(p*, u*) for left/right states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(200):
        fl, dl = _wave(p, rl, pl, cl, gamma)
        fr, dr = _wave(p, rr, pr, cr, gamma)
        g = fl + fr + (ur - ul)
        pn = max(1e-14, p - g / (dl + dr))
        if abs(pn - p) < tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _wave(p, rl, pl, cl, gamma)
    fr, _ = _wave(p, rr, pr, cr, gamma)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def sample(left, right, xi, gamma=1.4):
    """(rho, u, p) at similarity coordinate xi = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    out = np.empty((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                rs = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0)
                S = ul - cl * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
                out[:, n] = (rl, ul, pl) if s < S else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / gamma)
                cs = cl * (ps / pl) ** ((gamma - 1) / (2 * gamma))
                if s < ul - cl:
                    out[:, n] = (rl, ul, pl)
                elif s > us - cs:
                    out[:, n] = (rs, us, ps)
                else:
                    u = 2.0 / (gamma + 1) * (cl + 0.5 * (gamma - 1) * ul + s)
                    c = 2.0 / (gamma + 1) * (cl + 0.5 * (gamma - 1) * (ul - s))
                    r = rl * (c / cl) ** (2.0 / (gamma - 1))
                    out[:, n] = (r, u, pl * (c / cl) ** (2 * gamma / (gamma - 1)))
        else:  # right of the contact
            if ps > pr:  # right shock
                rs = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0)
                S = ur + cr * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
                out[:, n] = (rr, ur, pr) if s > S else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / gamma)
                cs = cr * (ps / pr) ** ((gamma - 1) / (2 * gamma))
                if s > ur + cr:
                    out[:, n] = (rr, ur, pr)
                elif s < us + cs:
                    out[:, n] = (rs, us, ps)
                else:
                    u = 2.0 / (gamma + 1) * (-cr + 0.5 * (gamma - 1) * ur + s)
                    c = 2.0 / (gamma + 1) * (cr - 0.5 * (gamma - 1) * (ur - s))
                    r = rr * (c / cr) ** (2.0 / (gamma - 1))
                    out[:, n] = (r, u, pr * (c / cr) ** (2 * gamma / (gamma - 1)))
    return out


def solution(left, right, x, t, x0=0.5, gamma=1.4):
    return sample(left, right, (np.asarray(x) - x0) / t, gamma)
