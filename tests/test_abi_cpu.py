"""The C-ABI library builds, loads without a GPU and exports every function
include/pond.h declares; host-only entry points behave as documented."""
import ctypes
import os
import re

import pytest

from paper_2302_00310_gb300 import build as B
from paper_2302_00310_gb300 import pond

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, h)).read() for h in sorted(os.listdir(inc)) if h.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pond_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return pond.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(pond.EXPORTS) == names


def test_host_only_calls(L):
    assert pond.pond_abi_version() == 1
    p = pond.pond_params_default()
    assert p.gamma == 1.4 and p.cfl == 0.2 and p.iter_max == 10
    assert pond.pond_strerror(pond.POND_E_NONPHYSICAL).startswith("nonphysical")
    n1 = pond.pond_workspace_size(pond.POND_D2Q16, (256, 256), p)
    assert n1 >= 2 * 256 * 256 * 28 * 8
    p.precision = pond.POND_FP32_MIXED
    n2 = pond.pond_workspace_size(pond.POND_D2Q16, (256, 256), p)
    assert n2 < n1


def test_invalid_arguments_are_rejected_before_any_device_work(L):
    p = pond.pond_params_default()
    with pytest.raises(pond.PondError) as e:
        pond.pond_workspace_size(pond.POND_D2Q16, (1, 8), p)
    assert e.value.status == pond.POND_E_INVAL
    p.tau = -1.0
    with pytest.raises(pond.PondError) as e:
        pond.pond_create(pond.POND_D2Q16, (8, 8), p)
    assert e.value.status == pond.POND_E_INVAL
    p = pond.pond_params_default()
    p.bc[0] = pond.POND_BC_PERIODIC
    p.bc[1] = pond.POND_BC_ZERO_GRADIENT
    with pytest.raises(pond.PondError):
        pond.pond_create(pond.POND_D2Q16, (8, 8), p)
    with pytest.raises(pond.PondError):
        pond.pond_create(7, (8, 8), pond.pond_params_default())


def _params(**kw):
    p = pond.pond_params_default()
    for k, v in kw.items():
        if k == "bc":
            for i, b in enumerate(v):
                p.bc[i] = b
        else:
            setattr(p, k, v)
    return p


@pytest.mark.parametrize("lat,kw", [
    # multiscale: averaged frame, no D2Q25, the precision's tile, App. C when mixed
    (pond.POND_D2Q16, dict(multiscale=1, flux_frame=pond.POND_FRAME_ITER)),
    (pond.POND_D2Q25, dict(multiscale=1)),
    (pond.POND_D2Q16, dict(multiscale=1, tile=6)),
    (pond.POND_D2Q16, dict(multiscale=2)),
    (pond.POND_D2Q16, dict(multiscale=1, ms_theta_u=float("nan"))),
    # g on the f-lattice: no D2Q25, no multiscale, averaged frame, the precision's tile
    (pond.POND_D2Q25, dict(g_same_as_f=1)),
    (pond.POND_D2Q16, dict(g_same_as_f=1, multiscale=1)),
    (pond.POND_D2Q16, dict(g_same_as_f=1, flux_frame=pond.POND_FRAME_ITER)),
    (pond.POND_D2Q16, dict(g_same_as_f=1, tile=9)),
    # tile 11 (8x14 capped for three CTAs per SM) is a mixed-path shape
    (pond.POND_D2Q16, dict(tile=11)),
    (pond.POND_D2Q16, dict(tile=12, precision=pond.POND_FP32_MIXED)),
    (pond.POND_D2Q16, dict(g_same_as_f=1, precision=pond.POND_FP32_MIXED, tile=6)),
    (pond.POND_D1Q4, dict(g_same_as_f=2)),
])
def test_multiscale_and_g_lattice_combinations_are_rejected_before_any_device_work(L, lat, kw):
    with pytest.raises(pond.PondError) as e:
        pond.pond_create(lat, (16, 16), _params(**kw))
    assert e.value.status == pond.POND_E_INVAL


def test_g_on_the_f_lattice_sizes_the_workspace_for_its_populations(L):
    n3 = pond.pond_workspace_size(pond.POND_D2Q16, (64, 64), _params())
    n4 = pond.pond_workspace_size(pond.POND_D2Q16, (64, 64), _params(g_same_as_f=1))
    assert n4 - n3 >= 2 * 64 * 64 * (16 - 9) * 8


def test_batch_tile_codes_are_resolved_before_any_device_work(L):
    """pond_batch_create resolves the requested tile among the candidates of
    the batch's precision before its first CUDA call: a candidate gets as far
    as the device query (POND_E_CUDA without a GPU), anything else is
    POND_E_INVAL; a zero tile (autotune) resolves too."""
    import ctypes

    import torch

    no_gpu = not torch.cuda.is_available()
    for prec, tile, ok in ((pond.POND_FP64, 9, True), (pond.POND_FP64, 10, True),
                           (pond.POND_FP64, 4, False), (pond.POND_FP32_MIXED, 10, True),
                           (pond.POND_FP32_MIXED, 11, True), (pond.POND_FP64, 11, False),
                           (pond.POND_FP32_MIXED, 6, True), (pond.POND_FP32_MIXED, 3, False),
                           (pond.POND_FP32_MIXED, 4, False), (pond.POND_FP32_MIXED, 9, False),
                           (pond.POND_FP64, 0, True), (pond.POND_FP32_MIXED, 0, True)):
        t = pond.pond_tune_default()
        t.tile = tile
        b = ctypes.c_void_p()
        st = L.pond_batch_create(ctypes.byref(b), 2, prec, 4, ctypes.byref(t), None)
        if not ok:
            assert st == pond.POND_E_INVAL, (prec, tile, st)
        elif no_gpu:
            assert st == pond.POND_E_CUDA, (prec, tile, st)
        else:
            assert st == pond.POND_OK
            L.pond_batch_destroy(b)


def test_noalloc_refuses_host_arrays(L):
    """pond_step_noalloc has no host-memory path: numpy arrays are refused in
    the binding, before the C call could treat them as device addresses."""
    import numpy as np

    p = pond.pond_params_default()
    p.dt = 1e-4
    a = np.zeros(64)
    with pytest.raises(TypeError):
        pond.pond_step_noalloc(pond.POND_D1Q4, (16, 1), p, a, a, a, None, a, 1)
