"""FP64 CPU oracle of the Particles-on-Demand time step (arXiv:2302.00310).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The product
library never calls it, and it shares no code with the CUDA path: the
arithmetic lives in ``pond_oracle.c`` (plain C, every value a double, one
explicit frame transformation per stencil cell per face), and this module only
marshals numpy arrays through ctypes.

Array layouts follow the product's state layout so that results compare
element by element: populations ``[i][ny][nx]`` with ``i = iy*q + ix`` (x
fastest), fields ``[ny][nx]``; a 1D run has ``ny = 1``.

Parity status: every exported function is pinned by ``tests/test_oracle_*.py``
against values the paper and the mathematics fix (Table I moments, Appendix A
closed forms, the Appendix B matrix form, Maxwell-Boltzmann moments of Sec.
II.D, the frame-variance deviation R', conservation, Galilean invariance of a
uniform state, the exact Riemann solution of the Sod problem, and an
independent multi-precision restatement of one step on tiny grids).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pond_oracle.c")
_SO = os.path.join(_HERE, "libpond_oracle.so")
# the same source with its operation counters compiled in (count_ops only)
_SO_COUNT = os.path.join(_HERE, "libpond_oracle_count.so")

BC_PERIODIC, BC_ZERO_GRADIENT, BC_INFLOW, BC_WALL = 0, 1, 2, 3
LIM_VANLEER, LIM_MINMOD = 0, 1
FLAG_NONPHYSICAL, FLAG_NOCONV = 1, 4


def _compile(so: str, defines, force: bool) -> str:
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(_SRC):
        return so
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("oracle: no C compiler found")
    base = [cc, "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"] + defines
    tmp = so + ".tmp"
    for extra in (["-fopenmp"], []):
        cmd = base + extra + ["-o", tmp, _SRC, "-lm"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(tmp, so)
            return so
    raise RuntimeError("oracle: compile failed:\n" + r.stderr)


def build(force: bool = False) -> str:
    """Compile ``pond_oracle.c`` into ``libpond_oracle.so`` (gcc, -O2, strict
    FP: no contraction, so the arithmetic is exactly the source's), and the
    same source with its operation counters into ``libpond_oracle_count.so``."""
    _compile(_SO_COUNT, ["-DORC_COUNT_OPS"], force)
    return _compile(_SO, [], force)


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
        d = ctypes.c_double
        P = ctypes.POINTER(ctypes.c_double)
        _lib.orc_lattice.argtypes = [ctypes.c_int, P, P]
        _lib.orc_lattice.restype = ctypes.c_int
        _lib.orc_transform_pub.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, d, P, d, P]
        _lib.orc_transform_x_pub.argtypes = [ctypes.c_int] * 5 + [P, P, d, P, d, P]
        _lib.orc_equilibrium_pub.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, d, P, d, P, d, P]
        _lib.orc_qe_half_pub.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, d, d, d, d, P, P, P, d]
        _lib.orc_macro_pub.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, d, P, P, P, d, P]
        _lib.orc_macro_pub.restype = ctypes.c_int
        _lib.orc_init.argtypes = [ctypes.c_void_p] + [P] * 9
        _lib.orc_init.restype = ctypes.c_int
        _lib.orc_run.argtypes = [ctypes.c_void_p, P, P, P, P, P, ctypes.c_int64, ctypes.c_void_p]
        _lib.orc_ghost_pub.argtypes = [ctypes.c_void_p] + [P] * 5 + [ctypes.c_int] * 2 + [P] * 3
        _lib.orc_ghost_pub.restype = ctypes.c_int
        _lib.orc_ms_measure_pub.argtypes = [ctypes.c_void_p] + [P] * 5
        _lib.orc_ms_measure_pub.restype = ctypes.c_int
        _lib.orc_run.restype = ctypes.c_int
        _lib.orc_threads.restype = ctypes.c_int
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib.orc_set_threads.restype = None
    return _lib


_lib_count = None


def _counting_lib():
    global _lib_count
    if _lib_count is None:
        build()
        _lib_count = ctypes.CDLL(_SO_COUNT)
        P = ctypes.POINTER(ctypes.c_double)
        _lib_count.orc_count_ops.argtypes = [ctypes.c_void_p, P, P, P, P, P, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]
        _lib_count.orc_count_ops.restype = ctypes.c_int
    return _lib_count


class _Params(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("qf", ctypes.c_int), ("qg", ctypes.c_int),
        ("gamma", ctypes.c_double), ("tau", ctypes.c_double), ("prandtl", ctypes.c_double),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("bc", ctypes.c_int * 4), ("inflow", (ctypes.c_double * 4) * 4),
        ("grad_k", ctypes.c_int), ("flux_appc", ctypes.c_int), ("limiter", ctypes.c_int),
        ("iterative", ctypes.c_int), ("iter_tol", ctypes.c_double), ("iter_max", ctypes.c_int),
        ("ms", ctypes.c_int), ("ms_theta_u", ctypes.c_double), ("ms_theta_T", ctypes.c_double),
    ]


class _Report(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("noconv_faces", ctypes.c_int64),
                ("max_cfl", ctypes.c_double), ("face_evals", ctypes.c_int64),
                ("traces", ctypes.c_int64), ("max_traces", ctypes.c_int32),
                ("ms_high", ctypes.c_int64)]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(x, n=2):
    v = np.zeros(n, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    v[: x.size] = x
    return v


def lattice(q: int):
    """Nodes, weights and invariant order of the q-node 1D lattice (Table I)."""
    c = np.zeros(5)
    w = np.zeros(5)
    K = lib().orc_lattice(q, _ptr(c), _ptr(w))
    return c[:q].copy(), w[:q].copy(), K


def transform(q, D, fin, u, T, up, Tp, grad_k=0):
    """Frame transformation G_{u,T}^{up,Tp} of one population vector."""
    fin = np.ascontiguousarray(fin, dtype=np.float64)
    out = np.zeros(q**D)
    lib().orc_transform_pub(q, D, int(grad_k), _ptr(fin), _ptr(_vec(u)), float(T),
                            _ptr(_vec(up)), float(Tp), _ptr(out))
    return out


def transform_x(qs, qd, K, D, fin, u, T, up, Tp, grad_k=0):
    """Frame transformation from the qs-node lattice in (u, T) to the qd-node
    lattice in (up, Tp), keeping coefficients of order <= K per axis
    (multiscale lifting or projection)."""
    fin = np.ascontiguousarray(fin, dtype=np.float64)
    out = np.zeros(qd**D)
    lib().orc_transform_x_pub(qs, qd, int(K), D, int(grad_k), _ptr(fin), _ptr(_vec(u)), float(T),
                              _ptr(_vec(up)), float(Tp), _ptr(out))
    return out


def equilibrium(q, D, rho, u, T, up, Tp, grad_k=0):
    """rho G_{u,T}^{up,Tp} W: equilibrium of (rho, u, T) written in frame (up, Tp)."""
    out = np.zeros(q**D)
    lib().orc_equilibrium_pub(q, D, int(grad_k), float(rho), _ptr(_vec(u)), float(T),
                              _ptr(_vec(up)), float(Tp), _ptr(out))
    return out


def qe_half(qf, qg, D, gamma, dt, tau1, tau2, f, g, u, T):
    """One quasi-equilibrium half relaxation of a cell (returns new f, g)."""
    f = np.array(f, dtype=np.float64)
    g = np.array(g, dtype=np.float64)
    lib().orc_qe_half_pub(qf, qg, D, float(gamma), float(dt), float(tau1), float(tau2),
                          _ptr(f), _ptr(g), _ptr(_vec(u)), float(T))
    return f, g


def macro(qf, qg, D, gamma, f, g, uf, Tf):
    """(rho, ux, uy, T) of one cell whose populations are given in frame (uf, Tf)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(4)
    ok = lib().orc_macro_pub(qf, qg, D, float(gamma), _ptr(f), _ptr(g), _ptr(_vec(uf)), float(Tf),
                             _ptr(out))
    return out, bool(ok)


@dataclass
class Config:
    """Run parameters of the oracle (its own mirror of a run configuration)."""
    D: int
    nx: int
    ny: int = 1
    qf: int = 4
    qg: int = 3
    gamma: float = 1.4
    tau: float = 1e-3
    prandtl: float = 1.0
    dx: float = 1.0
    dt: float = 1e-3
    bc: tuple = (BC_ZERO_GRADIENT,) * 4
    inflow: tuple = ((0.0,) * 4,) * 4
    grad_k: int = 0
    flux_appc: int = 0
    limiter: int = LIM_VANLEER
    iterative: int = 0
    iter_tol: float = 1e-12
    iter_max: int = 10
    ms: int = 0
    ms_theta_u: float = 0.0
    ms_theta_T: float = 0.0

    @classmethod
    def from_dict(cls, d: dict) -> "Config":
        names = {f for f in cls.__dataclass_fields__}
        return cls(**{k: v for k, v in d.items() if k in names})

    def _c(self) -> _Params:
        p = _Params()
        p.D, p.nx, p.ny = self.D, self.nx, (self.ny if self.D == 2 else 1)
        p.qf, p.qg = self.qf, self.qg
        p.gamma, p.tau, p.prandtl = self.gamma, self.tau, self.prandtl
        p.dx, p.dt = self.dx, self.dt
        for s in range(4):
            p.bc[s] = int(self.bc[s])
            for m in range(4):
                p.inflow[s][m] = float(self.inflow[s][m])
        p.grad_k, p.flux_appc, p.limiter = int(self.grad_k), int(self.flux_appc), int(self.limiter)
        p.iterative, p.iter_tol, p.iter_max = int(self.iterative), float(self.iter_tol), int(self.iter_max)
        p.ms, p.ms_theta_u, p.ms_theta_T = int(self.ms), float(self.ms_theta_u), float(self.ms_theta_T)
        return p


@dataclass
class State:
    """Populations f [Qf, ny, nx], g [Qg, ny, nx] in each cell's co-moving frame,
    and the frame (ux, uy, T), each [ny, nx]."""
    f: np.ndarray
    g: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    T: np.ndarray
    report: dict = field(default_factory=dict)

    def copy(self) -> "State":
        return State(self.f.copy(), self.g.copy(), self.ux.copy(), self.uy.copy(), self.T.copy(),
                     dict(self.report))


def init(cfg: Config, rho, ux, uy, T) -> State:
    """Co-moving equilibrium state (Eqs. feqPond, geqPond) from primitive fields."""
    ny = cfg.ny if cfg.D == 2 else 1
    shp = (ny, cfg.nx)
    arr = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64).reshape(-1)
                                                if np.ndim(a) else a, (ny * cfg.nx,)).reshape(shp))
           for a in (rho, ux, uy, T)]
    Qf, Qg = cfg.qf**cfg.D, cfg.qg**cfg.D
    st = State(np.zeros((Qf,) + shp), np.zeros((Qg,) + shp), np.zeros(shp), np.zeros(shp),
               np.zeros(shp))
    rc = lib().orc_init(ctypes.byref(cfg._c()), *[_ptr(a) for a in arr],
                        _ptr(st.f), _ptr(st.g), _ptr(st.ux), _ptr(st.uy), _ptr(st.T))
    if rc != 0:
        raise ValueError("oracle: invalid configuration")
    return st


def run(cfg: Config, state: State, nsteps: int) -> State:
    """Advance a copy of ``state`` by ``nsteps`` PonD steps."""
    st = state.copy()
    rep = _Report()
    rc = lib().orc_run(ctypes.byref(cfg._c()), _ptr(st.f), _ptr(st.g), _ptr(st.ux), _ptr(st.uy),
                       _ptr(st.T), int(nsteps), ctypes.byref(rep))
    if rc != 0:
        raise ValueError("oracle: invalid configuration (rc=%d)" % rc)
    st.report = {"flags": int(rep.flags), "noconv_faces": int(rep.noconv_faces),
                 "max_cfl": float(rep.max_cfl), "face_evals": int(rep.face_evals),
                 "traces": int(rep.traces), "max_traces": int(rep.max_traces),
                 "ms_high": int(rep.ms_high)}
    return st


def count_ops(cfg: Config, state: State, nsteps: int):
    """Floating-point operations (+, -, *, /, sqrt) of ``nsteps`` oracle steps
    from ``state`` on one thread, and the advanced copy: the stages of the step
    on cells and faces, not the construction of ghost cells."""
    st = state.copy()
    rep = _Report()
    ops = ctypes.c_int64()
    rc = _counting_lib().orc_count_ops(ctypes.byref(cfg._c()), _ptr(st.f), _ptr(st.g), _ptr(st.ux),
                                       _ptr(st.uy), _ptr(st.T), int(nsteps), ctypes.byref(rep),
                                       ctypes.byref(ops))
    if rc != 0:
        raise ValueError("oracle: invalid configuration (rc=%d)" % rc)
    return int(ops.value), st


def ms_measure(cfg: Config, ux, uy, T):
    """Multiscale switching measures (s_u, s_T), each [ny, nx], of the fields
    under the run's boundary rules (a cell takes the high lattice where
    s_u > ms_theta_u or s_T > ms_theta_T)."""
    ny = cfg.ny if cfg.D == 2 else 1
    shp = (ny, cfg.nx)
    arr = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), shp))
           for a in (ux, uy, T)]
    su, sT = np.zeros(shp), np.zeros(shp)
    rc = lib().orc_ms_measure_pub(ctypes.byref(cfg._c()), *[_ptr(a) for a in arr], _ptr(su), _ptr(sT))
    if rc != 0:
        raise ValueError("oracle: invalid configuration")
    return su, sT


def ghost(cfg: Config, st: State, j: int, k: int):
    """The ghost cell (j, k) (up to two layers beyond the interior) that the
    run's boundary rules build from ``st``: (f[Qf], g[Qg], (ux, uy, T))."""
    f = np.zeros(cfg.qf**cfg.D)
    g = np.zeros(cfg.qg**cfg.D)
    fr = np.zeros(3)
    rc = lib().orc_ghost_pub(ctypes.byref(cfg._c()), _ptr(st.f), _ptr(st.g), _ptr(st.ux),
                             _ptr(st.uy), _ptr(st.T), int(j), int(k), _ptr(f), _ptr(g), _ptr(fr))
    if rc != 0:
        raise ValueError("oracle: invalid configuration or not a ghost cell (rc=%d)" % rc)
    return f, g, tuple(fr)


def moments(cfg: Config, st: State):
    """rho, ux, uy, T fields recomputed from the populations (each cell in its frame)."""
    ny = cfg.ny if cfg.D == 2 else 1
    out = np.zeros((4, ny, cfg.nx))
    for k in range(ny):
        for j in range(cfg.nx):
            o, _ = macro(cfg.qf, cfg.qg, cfg.D, cfg.gamma, st.f[:, k, j], st.g[:, k, j],
                         (st.ux[k, j], st.uy[k, j]), st.T[k, j])
            out[:, k, j] = o
    return out


def threads() -> int:
    return int(lib().orc_threads())


def set_threads(n: int) -> None:
    """OpenMP threads for later oracle runs."""
    lib().orc_set_threads(int(n))
