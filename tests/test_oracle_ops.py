"""The oracle's operation counter (the work the step's stages do on cells and
faces, as the oracle computes them; ghost construction excluded).  Pins:

* counting changes no arithmetic: the counted run's state is the plain run's,
  bit for bit;
* on a uniform periodic flow every cell and face does the same work each step,
  so the count is exactly linear in the steps and a polynomial of degree D in
  the grid's side: D + 1 sizes fix it and one more is predicted exactly;
* van Leer costs more than minmod by 4 operations per limited slope, and on a
  uniform flow no slope is limited, so there the two counts agree.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2302_00310_gb300 import workloads as W


def _uniform(D, n, limiter=0, qf=4):
    shp = (n if D == 2 else 1, n)
    rho, T = np.full(shp, 1.1), np.full(shp, 0.8)
    ux, uy = np.full(shp, 0.7), np.full(shp, -0.4 if D == 2 else 0.0)
    d = W._base(D, n, n, qf=qf, tau=1e-3, dx=1.0 / n, limiter=limiter, bc=(0, 0, 0, 0))
    d["dt"] = W.dt_from_cfl(ux, uy, T, d["dx"], 0.3)
    cfg = oracle.Config.from_dict(d)
    return cfg, oracle.init(cfg, rho, ux, uy, T)


def test_counting_changes_no_arithmetic():
    w = W.pulse_2d(n=24, seed=2)
    cfg = oracle.Config.from_dict(w["cfg"])
    st = oracle.init(cfg, w["rho"], w["ux"], w["uy"], w["T"])
    ops, counted = oracle.count_ops(cfg, st, 2)
    plain = oracle.run(cfg, st, 2)
    assert ops > 0
    assert np.array_equal(counted.f, plain.f) and np.array_equal(counted.g, plain.g)
    assert np.array_equal(counted.T, plain.T)


@pytest.mark.parametrize("D", [1, 2])
def test_uniform_flow_count_is_polynomial_in_the_side(D):
    """Each interior cell, each face and each padded cell (phi_bar^+ is built
    on the ghosts too) does fixed work, plus a fixed amount per step: the count
    of one step is a polynomial of degree D in the side n.  D + 1 sizes fix it,
    and one more size is predicted exactly."""
    sizes = (6, 8, 10, 12)[: D + 2]
    counts = []
    for n in sizes:
        cfg, st = _uniform(D, n)
        one, _ = oracle.count_ops(cfg, st, 1)
        three, _ = oracle.count_ops(cfg, st, 3)
        assert three == 3 * one
        counts.append(one)
    V = np.array([[float(n) ** k for k in range(D + 1)] for n in sizes[:-1]])
    coef = np.linalg.solve(V, np.array(counts[:-1], dtype=float))
    n = sizes[-1]
    predicted = sum(c * float(n) ** k for k, c in enumerate(coef))
    assert abs(predicted - counts[-1]) < 1e-6 * counts[-1]


def test_limiters_cost_the_same_where_nothing_is_limited():
    a, _ = oracle.count_ops(*_uniform(2, 6, limiter=oracle.LIM_VANLEER), 1)
    b, _ = oracle.count_ops(*_uniform(2, 6, limiter=oracle.LIM_MINMOD), 1)
    assert a == b
    w = W.pulse_2d(n=16, seed=4)
    for lim in (oracle.LIM_VANLEER, oracle.LIM_MINMOD):
        cfg = oracle.Config.from_dict(dict(w["cfg"], limiter=lim))
        st = oracle.init(cfg, w["rho"], w["ux"], w["uy"], w["T"])
        ops, _ = oracle.count_ops(cfg, st, 1)
        if lim == oracle.LIM_VANLEER:
            vl = ops
        else:
            mm = ops
    assert vl > mm and (vl - mm) % 4 == 0
