"""Thin ctypes binding of the C ABI in ``include/pond.h``.

Every function here marshals arguments and calls the function of the same
name in ``libpond_gb300.so``; all arithmetic of the time step runs in the
CUDA kernels behind it.  There is no CPU fallback: ``lib()`` raises if the
library has not been built.  PyTorch is used only for device memory and
streams (``Sim``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

POND_D1Q4, POND_D2Q16, POND_D2Q25 = 1, 2, 3
POND_OK, POND_E_INVAL, POND_E_NOMEM, POND_E_CUDA = 0, 1, 2, 3
POND_E_NONPHYSICAL, POND_E_NOCONV, POND_E_CFL, POND_E_STATE = 4, 5, 6, 7
POND_BC_PERIODIC, POND_BC_ZERO_GRADIENT, POND_BC_INFLOW = 0, 1, 2
POND_FP64, POND_FP32_MIXED = 0, 1
POND_TENSOR, POND_GRAD_K = 0, 1
POND_FLUX_MAIN, POND_FLUX_APPC = 0, 1
POND_VANLEER, POND_MINMOD = 0, 1
POND_FRAME_AVG, POND_FRAME_ITER = 0, 1
POND_FLAG_NONPHYSICAL, POND_FLAG_CFL, POND_FLAG_NOCONV = 1, 2, 4

# every symbol include/pond.h declares
EXPORTS = (
    "pond_params_default", "pond_workspace_size", "pond_create", "pond_init", "pond_step",
    "pond_moments", "pond_get_state", "pond_set_state", "pond_status_flags", "pond_reset_flags",
    "pond_iter_stats", "pond_ms_stats",
    "pond_sync", "pond_info", "pond_destroy", "pond_strerror", "pond_abi_version",
    "pond_step_noalloc", "pond_tune_default", "pond_batch_create", "pond_batch_add",
    "pond_batch_remove", "pond_batch_size", "pond_batch_step", "pond_batch_info",
    "pond_batch_destroy", "pond_checkpoint_size", "pond_checkpoint", "pond_restore",
    # include/pond_checks.h
    "pond_measure_fma_peak", "pond_check_reciprocal", "pond_check_vanleer",
)
POND_NOALLOC_SCRATCH_BYTES = 16 * 1024 * 1024


class pond_params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_double), ("tau", ctypes.c_double), ("prandtl", ctypes.c_double),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("cfl", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("inflow", (ctypes.c_double * 4) * 4),
        ("precision", ctypes.c_int32), ("transform", ctypes.c_int32),
        ("flux_form", ctypes.c_int32), ("limiter", ctypes.c_int32),
        ("flux_frame", ctypes.c_int32), ("iter_tol", ctypes.c_double),
        ("iter_max", ctypes.c_int32), ("xi_fp64_threshold", ctypes.c_double),
        ("tile", ctypes.c_int32), ("multiscale", ctypes.c_int32), ("ms_theta_u", ctypes.c_double),
        ("ms_theta_T", ctypes.c_double), ("g_same_as_f", ctypes.c_int32),
        ("strip", ctypes.c_int32),
    ]


class pond_tune(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("graph_steps", ctypes.c_int32),
                ("autotune", ctypes.c_int32)]


class PondError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, pond_strerror(status), status))


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def lib(build: bool = False):
    """Load ``libpond_gb300.so`` (building it first if ``build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libpond_gb300.so is not built (run __graft_entry__.build() or "
                           "python -m paper_2302_00310_gb300.build); there is no CPU fallback")
    L = ctypes.CDLL(_build.LIB)
    L.pond_params_default.argtypes = [ctypes.POINTER(pond_params)]
    L.pond_params_default.restype = None
    L.pond_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(pond_params), ctypes.POINTER(ctypes.c_size_t)]
    L.pond_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                              ctypes.POINTER(pond_params), _P, ctypes.c_size_t, _P]
    L.pond_init.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int]
    L.pond_step.argtypes = [_P, ctypes.c_int64]
    L.pond_moments.argtypes = [_P, _P, _P, _P, _P, ctypes.c_int]
    L.pond_get_state.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int]
    L.pond_set_state.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_int]
    L.pond_status_flags.argtypes = [_P, ctypes.POINTER(ctypes.c_uint32), _D,
                                    ctypes.POINTER(ctypes.c_int64)]
    L.pond_reset_flags.argtypes = [_P]
    L.pond_iter_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int32)]
    L.pond_ms_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
    L.pond_sync.argtypes = [_P]
    L.pond_info.argtypes = [_P, _D, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
    L.pond_destroy.argtypes = [_P]
    L.pond_destroy.restype = None
    L.pond_strerror.argtypes = [ctypes.c_int]
    L.pond_strerror.restype = ctypes.c_char_p
    L.pond_abi_version.restype = ctypes.c_int
    L.pond_step_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(pond_params), _P, _P, _P, _P, _P,
                                    ctypes.c_int64, ctypes.POINTER(ctypes.c_uint32), _P]
    L.pond_checkpoint_size.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t)]
    L.pond_checkpoint.argtypes = [_P, _P, ctypes.c_size_t]
    L.pond_restore.argtypes = [_P, _P, ctypes.c_size_t]
    L.pond_tune_default.argtypes = [ctypes.POINTER(pond_tune)]
    L.pond_tune_default.restype = None
    L.pond_batch_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_int32, ctypes.POINTER(pond_tune), _P]
    L.pond_batch_add.argtypes = [_P, _P]
    L.pond_batch_remove.argtypes = [_P, _P]
    L.pond_batch_size.argtypes = [_P]
    L.pond_batch_size.restype = ctypes.c_int32
    L.pond_batch_step.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
    L.pond_batch_info.argtypes = [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32), _D]
    L.pond_batch_destroy.argtypes = [_P]
    L.pond_batch_destroy.restype = None
    L.pond_measure_fma_peak.argtypes = [ctypes.c_int32, ctypes.c_double, _D, _D]
    L.pond_check_reciprocal.argtypes = [_P, _P, _P, ctypes.c_int64, _P]
    L.pond_check_vanleer.argtypes = [_P, _P, _P, _P, ctypes.c_int64, _P]
    no_status = ("pond_params_default", "pond_destroy", "pond_strerror", "pond_abi_version",
                 "pond_tune_default", "pond_batch_size", "pond_batch_destroy")
    for name in EXPORTS:
        if name not in no_status:
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int, what: str):
    if status != POND_OK:
        raise PondError(status, what)


def _ptr(a):
    """Address of a contiguous FP64 host array or CUDA tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous, "need contiguous float64"
        return a.ctypes.data
    assert a.is_contiguous() and str(a.dtype) == "torch.float64", "need contiguous float64 tensor"
    return a.data_ptr()


def _on_device(*arrays) -> int:
    dev = [not isinstance(a, np.ndarray) for a in arrays if a is not None]
    assert all(dev) or not any(dev), "mix of host and device arrays"
    return int(bool(dev) and dev[0])


# ---- the ABI, same names ------------------------------------------------------
def pond_strerror(status: int) -> str:
    return lib().pond_strerror(int(status)).decode()


def pond_abi_version() -> int:
    return int(lib().pond_abi_version())


def pond_params_default() -> pond_params:
    p = pond_params()
    lib().pond_params_default(ctypes.byref(p))
    return p


def pond_workspace_size(lat: int, dims, params: pond_params) -> int:
    d = (ctypes.c_int64 * 2)(*[int(x) for x in dims])
    out = ctypes.c_size_t()
    _check(lib().pond_workspace_size(int(lat), d, ctypes.byref(params), ctypes.byref(out)),
           "pond_workspace_size")
    return int(out.value)


def pond_create(lat: int, dims, params: pond_params, workspace: int | None = None,
                workspace_bytes: int = 0, stream: int | None = None):
    d = (ctypes.c_int64 * 2)(*[int(x) for x in dims])
    ctx = _P()
    _check(lib().pond_create(ctypes.byref(ctx), int(lat), d, ctypes.byref(params), workspace,
                             int(workspace_bytes), stream), "pond_create")
    return ctx


def pond_init(ctx, rho, ux, uy, T):
    _check(lib().pond_init(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T),
                           _on_device(rho, ux, uy, T)), "pond_init")


class nvtx_range:
    """An NVTX range (visible in Nsight timelines) around host calls that
    enqueue steps; a no-op where PyTorch's NVTX bindings are unavailable."""

    def __init__(self, name: str):
        self.name = name
        self._nvtx = None

    def __enter__(self):
        try:
            import torch

            torch.cuda.nvtx.range_push(self.name)
            self._nvtx = torch.cuda.nvtx
        except Exception:
            self._nvtx = None
        return self

    def __exit__(self, *exc):
        if self._nvtx is not None:
            self._nvtx.range_pop()
        return False


def pond_step(ctx, n: int):
    _check(lib().pond_step(ctx, int(n)), "pond_step")


def pond_moments(ctx, rho, ux, uy, T):
    _check(lib().pond_moments(ctx, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T),
                              _on_device(rho, ux, uy, T)), "pond_moments")


def pond_get_state(ctx, f, g, ux, uy, T):
    _check(lib().pond_get_state(ctx, _ptr(f), _ptr(g), _ptr(ux), _ptr(uy), _ptr(T),
                                _on_device(f, g, ux, uy, T)), "pond_get_state")


def pond_set_state(ctx, f, g, ux, uy, T):
    _check(lib().pond_set_state(ctx, _ptr(f), _ptr(g), _ptr(ux), _ptr(uy), _ptr(T),
                                _on_device(f, g, ux, uy, T)), "pond_set_state")


def pond_status_flags(ctx):
    """(status, flags, max_cfl, noconv_faces); status is POND_E_NONPHYSICAL
    when that flag is set."""
    fl = ctypes.c_uint32()
    cfl = ctypes.c_double()
    nc = ctypes.c_int64()
    st = lib().pond_status_flags(ctx, ctypes.byref(fl), ctypes.byref(cfl), ctypes.byref(nc))
    if st not in (POND_OK, POND_E_NONPHYSICAL):
        raise PondError(st, "pond_status_flags")
    return st, int(fl.value), float(cfl.value), int(nc.value)


def pond_iter_stats(ctx):
    """(face evaluations, traces, most traces at one face) of the iterated
    face frame since the last reset."""
    ev, tr, mx = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
    _check(lib().pond_iter_stats(ctx, ctypes.byref(ev), ctypes.byref(tr), ctypes.byref(mx)),
           "pond_iter_stats")
    return int(ev.value), int(tr.value), int(mx.value)


def pond_ms_stats(ctx):
    """Cell updates made on the high-order f-lattice since the last reset
    (multiscale)."""
    n = ctypes.c_int64()
    _check(lib().pond_ms_stats(ctx, ctypes.byref(n)), "pond_ms_stats")
    return int(n.value)


def pond_reset_flags(ctx):
    _check(lib().pond_reset_flags(ctx), "pond_reset_flags")


def pond_sync(ctx):
    _check(lib().pond_sync(ctx), "pond_sync")


def pond_info(ctx):
    dt = ctypes.c_double()
    steps = ctypes.c_int64()
    tile = ctypes.c_int32()
    _check(lib().pond_info(ctx, ctypes.byref(dt), ctypes.byref(steps), ctypes.byref(tile)),
           "pond_info")
    return float(dt.value), int(steps.value), int(tile.value)


def pond_destroy(ctx):
    if ctx:
        lib().pond_destroy(ctx)


def pond_step_noalloc(lat: int, dims, params: pond_params, f, g, ux, uy, T, n: int,
                      stream: int | None = None, want_flags: bool = True):
    """FP64 steps of a caller-owned device state (CUDA tensors), in place, with
    no device allocation; returns (status, flags) (flags None if not wanted).

    Every array must be a contiguous float64 CUDA tensor (uy may be None in
    1D): the C call has no host-memory path, so a host array is refused here
    with TypeError rather than handed to the kernels as a device address."""
    for name, a in (("f", f), ("g", g), ("ux", ux), ("uy", uy), ("T", T)):
        if a is None and name == "uy" and int(lat) == POND_D1Q4:
            continue
        if (a is None or isinstance(a, np.ndarray) or not getattr(a, "is_cuda", False)
                or str(a.dtype) != "torch.float64" or not a.is_contiguous()):
            raise TypeError("pond_step_noalloc: %s must be a contiguous float64 CUDA tensor" % name)
    d = (ctypes.c_int64 * 2)(*[int(x) for x in dims])
    fl = ctypes.c_uint32()
    st = lib().pond_step_noalloc(int(lat), d, ctypes.byref(params), _ptr(f), _ptr(g), _ptr(ux),
                                 _ptr(uy), _ptr(T), int(n),
                                 ctypes.byref(fl) if want_flags else None, stream)
    if st not in (POND_OK, POND_E_NONPHYSICAL):
        raise PondError(st, "pond_step_noalloc")
    return st, (int(fl.value) if want_flags else None)


def pond_measure_fma_peak(precision: int, min_seconds: float = 0.5):
    """(TFLOP/s, ms of the best launch) of independent fma chains in FP64
    (POND_FP64) or FP32 (POND_FP32_MIXED) on the current device."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().pond_measure_fma_peak(int(precision), float(min_seconds), ctypes.byref(tf),
                                       ctypes.byref(ms)), "pond_measure_fma_peak")
    return float(tf.value), float(ms.value)


def _dev_f64(a, name):
    if isinstance(a, np.ndarray) or not getattr(a, "is_cuda", False) or \
            str(a.dtype) != "torch.float64" or not a.is_contiguous():
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    return a.data_ptr()


def pond_check_reciprocal(y, r, r_ref, stream: int | None = None):
    """The kernels' FP64 reciprocal of y into r, CUDA's __drcp_rn into r_ref."""
    _check(lib().pond_check_reciprocal(_dev_f64(y, "y"), _dev_f64(r, "r"), _dev_f64(r_ref, "r_ref"),
                                       int(y.numel()), stream), "pond_check_reciprocal")


def pond_check_vanleer(x, y, l, l_ref, stream: int | None = None):
    """The kernels' FP64 van Leer limiter of (x, y) into l, the same with
    CUDA's division into l_ref."""
    _check(lib().pond_check_vanleer(_dev_f64(x, "x"), _dev_f64(y, "y"), _dev_f64(l, "l"),
                                    _dev_f64(l_ref, "l_ref"), int(x.numel()), stream),
           "pond_check_vanleer")


def pond_checkpoint_size(ctx) -> int:
    n = ctypes.c_size_t()
    _check(lib().pond_checkpoint_size(ctx, ctypes.byref(n)), "pond_checkpoint_size")
    return int(n.value)


def pond_checkpoint(ctx) -> np.ndarray:
    """The context's checkpoint as a host byte array."""
    buf = np.empty(pond_checkpoint_size(ctx), dtype=np.uint8)
    _check(lib().pond_checkpoint(ctx, buf.ctypes.data, buf.nbytes), "pond_checkpoint")
    return buf


def pond_restore(ctx, buf: np.ndarray):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().pond_restore(ctx, buf.ctypes.data, buf.nbytes), "pond_restore")


def pond_tune_default() -> pond_tune:
    t = pond_tune()
    lib().pond_tune_default(ctypes.byref(t))
    return t


def pond_batch_create(dim: int, precision: int, capacity: int, tune: pond_tune | None = None,
                      stream: int | None = None):
    b = _P()
    _check(lib().pond_batch_create(ctypes.byref(b), int(dim), int(precision), int(capacity),
                                   ctypes.byref(tune) if tune is not None else None, stream),
           "pond_batch_create")
    return b


def pond_batch_add(b, ctx):
    _check(lib().pond_batch_add(b, ctx), "pond_batch_add")


def pond_batch_remove(b, ctx):
    _check(lib().pond_batch_remove(b, ctx), "pond_batch_remove")


def pond_batch_size(b) -> int:
    return int(lib().pond_batch_size(b))


def pond_batch_step(b, steps=None):
    """steps: one count per member (in the order they were added), or None
    for one step each."""
    arr = None
    if steps is not None:
        arr = (ctypes.c_int64 * len(steps))(*[int(x) for x in steps])
    _check(lib().pond_batch_step(b, arr), "pond_batch_step")


def pond_batch_info(b):
    """(tile code, grid CTAs, tuned flag, MLUPS of the tuned chunk)."""
    tile, grid, tuned = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    ml = ctypes.c_double()
    _check(lib().pond_batch_info(b, ctypes.byref(tile), ctypes.byref(grid), ctypes.byref(tuned),
                                 ctypes.byref(ml)), "pond_batch_info")
    return int(tile.value), int(grid.value), bool(tuned.value), float(ml.value)


def pond_batch_destroy(b):
    if b:
        lib().pond_batch_destroy(b)


# ---- configuration ------------------------------------------------------------
def params_from_config(cfg: dict) -> pond_params:
    """pond_params from a run-configuration dict (see ``workloads``)."""
    p = pond_params_default()
    p.gamma, p.tau, p.prandtl = cfg["gamma"], cfg["tau"], cfg["prandtl"]
    p.dx, p.dt = cfg["dx"], cfg.get("dt", 0.0)
    p.cfl = cfg.get("cfl", 0.2)
    for s in range(4):
        p.bc[s] = int(cfg["bc"][s])
        for m in range(4):
            p.inflow[s][m] = float(cfg["inflow"][s][m])
    p.precision = int(cfg.get("precision", POND_FP64))
    p.transform = POND_GRAD_K if cfg.get("grad_k", 0) else POND_TENSOR
    p.flux_form = POND_FLUX_APPC if cfg.get("flux_appc", 0) else POND_FLUX_MAIN
    p.limiter = int(cfg.get("limiter", POND_VANLEER))
    p.flux_frame = POND_FRAME_ITER if cfg.get("iterative", 0) else POND_FRAME_AVG
    p.iter_tol, p.iter_max = float(cfg.get("iter_tol", 1e-12)), int(cfg.get("iter_max", 10))
    p.xi_fp64_threshold = float(cfg.get("xi_fp64_threshold", 8.0))
    p.tile = int(cfg.get("tile", 0))
    p.multiscale = int(cfg.get("ms", 0))
    p.ms_theta_u, p.ms_theta_T = float(cfg.get("ms_theta_u", 0.0)), float(cfg.get("ms_theta_T", 0.0))
    p.g_same_as_f = 1 if int(cfg.get("qg", 3)) == 4 else 0
    p.strip = int(cfg.get("strip", 0))
    return p


class Sim:
    """One PonD context whose device workspace is a PyTorch tensor and whose
    kernels run on a PyTorch CUDA stream."""

    def __init__(self, cfg: dict, stream=None, device=None):
        import torch

        self.cfg = dict(cfg)
        self.D = int(cfg["D"])
        self.q1 = int(cfg.get("qf", 4))  # f nodes per axis: 4, or 5 for D2Q25
        self.lat = (POND_D2Q25 if self.q1 == 5 else POND_D2Q16) if self.D == 2 else POND_D1Q4
        self.nx = int(cfg["nx"])
        self.ny = int(cfg["ny"]) if self.D == 2 else 1
        self.params = params_from_config(cfg)
        self.device = torch.device(device or "cuda")
        # a stream of its own: consecutive steps are replayed from a captured graph
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        nbytes = pond_workspace_size(self.lat, (self.nx, self.ny), self.params)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.ctx = pond_create(self.lat, (self.nx, self.ny), self.params, aligned, nbytes,
                               self.stream.cuda_stream)

    @property
    def shape(self):
        return (self.ny, self.nx)

    @property
    def Qf(self):
        return self.q1 * self.q1 if self.D == 2 else 4

    @property
    def Qg(self):
        q = 4 if int(self.cfg.get("qg", 3)) == 4 else 3
        return q * q if self.D == 2 else q

    def init(self, rho, ux, uy, T):
        a = [np.ascontiguousarray(np.broadcast_to(np.asarray(x, dtype=np.float64), self.shape))
             if not hasattr(x, "data_ptr") else x for x in (rho, ux, uy, T)]
        pond_init(self.ctx, a[0], a[1], a[2] if self.D == 2 else None, a[3])

    def step(self, n: int):
        with nvtx_range("pond_step"):
            pond_step(self.ctx, n)

    def moments(self):
        out = [np.zeros(self.shape) for _ in range(4)]
        pond_moments(self.ctx, out[0], out[1], out[2] if self.D == 2 else None, out[3])
        return out

    def get_state(self):
        f = np.zeros((self.Qf,) + self.shape)
        g = np.zeros((self.Qg,) + self.shape)
        ux, uy, T = np.zeros(self.shape), np.zeros(self.shape), np.zeros(self.shape)
        pond_get_state(self.ctx, f, g, ux, uy if self.D == 2 else None, T)
        return f, g, ux, uy, T

    def set_state(self, f, g, ux, uy, T):
        c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        pond_set_state(self.ctx, c(f), c(g), c(ux), c(uy) if self.D == 2 else None, c(T))

    def flags(self):
        return pond_status_flags(self.ctx)

    def iter_stats(self):
        return pond_iter_stats(self.ctx)

    def ms_stats(self):
        return pond_ms_stats(self.ctx)

    def info(self):
        return pond_info(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            pond_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A pond_batch on a PyTorch stream, holding ``Sim`` members created on
    the same stream (``Sim(cfg, stream=batch.stream)``)."""

    def __init__(self, dim: int, precision: int, capacity: int, tune: pond_tune | None = None,
                 stream=None, device=None):
        import torch

        self.device = torch.device(device or "cuda")
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.members = []
        self.b = pond_batch_create(dim, precision, capacity, tune, self.stream.cuda_stream)

    def add(self, sim: "Sim"):
        pond_batch_add(self.b, sim.ctx)
        self.members.append(sim)

    def remove(self, sim: "Sim"):
        pond_batch_remove(self.b, sim.ctx)
        self.members.remove(sim)

    def step(self, steps=None):
        with nvtx_range("pond_batch_step"):
            pond_batch_step(self.b, steps)

    def info(self):
        return pond_batch_info(self.b)

    def close(self):
        if getattr(self, "b", None):
            pond_batch_destroy(self.b)
            self.b = None
            self.members = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
