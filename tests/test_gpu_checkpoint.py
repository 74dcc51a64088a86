"""Checkpoint / restore of a context's raw state: a run resumed from a
checkpoint continues bit for bit as the uninterrupted run."""
import numpy as np
import pytest

from paper_2302_00310_gb300 import pond
from paper_2302_00310_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pond.lib(build=True)


@pytest.mark.parametrize("D,precision", [(2, pond.POND_FP64), (2, pond.POND_FP32_MIXED),
                                         (1, pond.POND_FP64), (1, pond.POND_FP32_MIXED)])
def test_resume_is_bitwise_identical(D, precision):
    nx, ny = (37, 29) if D == 2 else (300, 1)
    prim = W.random_state_grid(D, nx, ny, seed=130, mach=0.8)
    cfg = W._base(D, nx, ny, tau=5e-3, dx=1.0 / nx, prandtl=0.71, bc=(1, 1, 0, 0),
                  precision=precision)
    cfg["dt"] = W.dt_from_cfl(prim[1], prim[2], prim[3], cfg["dx"], 0.4)
    a = pond.Sim(cfg)
    a.init(*prim)
    a.step(10)
    ck = pond.pond_checkpoint(a.ctx)
    a.step(17)
    want = a.get_state()
    info_a = a.info()
    a.close()
    b = pond.Sim(cfg)
    pond.pond_restore(b.ctx, ck)
    assert b.info()[1] == 10
    b.step(17)
    got = b.get_state()
    assert b.info()[:2] == info_a[:2]
    b.close()
    for x, y in zip(got, want):
        assert np.array_equal(x, y)


def test_restore_rejects_a_checkpoint_of_another_shape():
    prim = W.random_state_grid(2, 20, 20, seed=131, mach=0.5)
    cfg = W._base(2, 20, 20, tau=5e-3, dx=0.05, bc=(0, 0, 0, 0))
    cfg["dt"] = 1e-3
    a = pond.Sim(cfg)
    a.init(*prim)
    ck = pond.pond_checkpoint(a.ctx)
    a.close()
    for other in (dict(cfg, nx=21), dict(cfg, precision=pond.POND_FP32_MIXED)):
        b = pond.Sim(other)
        with pytest.raises(pond.PondError) as e:
            pond.pond_restore(b.ctx, ck)
        assert e.value.status == pond.POND_E_INVAL
        b.close()
    c = pond.Sim(cfg)
    bad = ck.copy()
    bad[0] ^= 0xFF
    with pytest.raises(pond.PondError):
        pond.pond_restore(c.ctx, bad)
    with pytest.raises(pond.PondError):
        pond.pond_restore(c.ctx, ck[:100])
    c.close()
