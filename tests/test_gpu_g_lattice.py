"""The g-populations on the f-lattice (pond_params.g_same_as_f: D1Q4 / D2Q16
for g instead of D1Q3 / D2Q9) on the GPU: the oracle's state with qg = 4 to
1e-12 in FP64 and the mixed path's moments within its step bound, across
tiles with ragged tails, boundaries (walls included), QE, both limiters,
Grad-K and Appendix C; and the configurations it does not cover."""
import numpy as np
import pytest

import oracle
from paper_2302_00310_gb300 import pond
from paper_2302_00310_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12
TOL_STEP = 2e-6
WALLS = ((0.0,) * 4, (0.0,) * 4, (0.0, 0.3, 0.0, 0.9), (0.0, -0.2, 0.0, 1.2))
INFLOW = ((1.1, 0.5, -0.2, 0.8),) * 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pond.lib(build=True)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


CASES = [
    # D, nx, ny, bc, prandtl, limiter, grad_k, appc, steps
    (2, 37, 30, (0, 0, 0, 0), 1.0, 0, 0, 0, 3),
    (2, 29, 33, (1, 1, 2, 1), 0.71, 1, 1, 0, 2),
    (2, 24, 31, (2, 1, 0, 0), 1.0, 0, 0, 1, 2),
    (2, 17, 23, (0, 0, 3, 3), 0.71, 1, 0, 0, 2),
    (1, 300, 1, (1, 1, 0, 0), 0.5, 0, 0, 0, 3),
    (1, 253, 1, (2, 1, 0, 0), 1.0, 1, 0, 1, 2),
]


def _cfg(case):
    D, nx, ny, bc, pr, lim, gk, appc, steps = case
    fields = W.random_state_grid(D, nx, ny, seed=170 + nx, mach=0.8, T=(0.7, 1.4))
    cfg = W._base(D, nx, ny, qg=4, tau=5e-3, dx=1.0 / nx, prandtl=pr, limiter=lim, grad_k=gk,
                  flux_appc=appc, bc=bc, inflow=WALLS if 3 in bc else INFLOW)
    cfg["dt"] = W.dt_from_cfl(fields[1], fields[2], fields[3], cfg["dx"], 0.4)
    return cfg, fields, steps


@pytest.mark.parametrize("case", range(len(CASES)))
def test_g_on_the_f_lattice_matches_oracle(case):
    cfg, fields, steps = _cfg(CASES[case])
    D = cfg["D"]
    ocfg = oracle.Config.from_dict(cfg)
    ost = oracle.run(ocfg, oracle.init(ocfg, *fields), steps)
    sim = pond.Sim(cfg)
    sim.init(*fields)
    sim.step(steps)
    f, g, ux, uy, T = sim.get_state()
    flags = sim.flags()
    sim.close()
    assert g.shape[0] == 4**D and ost.g.shape[0] == 4**D
    errs = {"f": _rel(f, ost.f), "g": _rel(g, ost.g), "ux": _rel(ux, ost.ux), "T": _rel(T, ost.T)}
    if D == 2:
        errs["uy"] = _rel(uy, ost.uy)
    assert max(errs.values()) <= TOL, errs
    assert flags[1] & pond.POND_FLAG_NONPHYSICAL == 0


@pytest.mark.parametrize("case", [0, 1, 3, 4])
def test_g_on_the_f_lattice_mixed_path(case):
    cfg, fields, steps = _cfg(CASES[case])
    ocfg = oracle.Config.from_dict(cfg)
    om = oracle.moments(ocfg, oracle.run(ocfg, oracle.init(ocfg, *fields), steps))
    sim = pond.Sim(dict(cfg, precision=pond.POND_FP32_MIXED))
    sim.init(*fields)
    sim.step(steps)
    gm = sim.moments()
    sim.close()
    for i in ((0, 1, 2, 3) if cfg["D"] == 2 else (0, 1, 3)):
        assert _rel(gm[i], om[i]) <= TOL_STEP, (i, _rel(gm[i], om[i]))


@pytest.mark.parametrize("bad", [dict(qf=5), dict(ms=1, ms_theta_u=0.1, ms_theta_T=0.1),
                                 dict(iterative=1), dict(tile=6)])
def test_g_on_the_f_lattice_rejects_what_it_does_not_cover(bad):
    fields = W.random_state_grid(2, 16, 16, seed=1)
    cfg = W._base(2, 16, 16, qg=4, tau=5e-3, dx=1.0 / 16)
    cfg["dt"] = 1e-4
    with pytest.raises(pond.PondError):
        sim = pond.Sim(dict(cfg, **bad))
        sim.init(*fields)
        sim.close()


def test_g_on_the_f_lattice_is_not_batched():
    fields = W.random_state_grid(2, 16, 16, seed=2)
    cfg = W._base(2, 16, 16, qg=4, tau=5e-3, dx=1.0 / 16)
    cfg["dt"] = 1e-4
    b = pond.Batch(2, pond.POND_FP64, 4)
    sim = pond.Sim(cfg, stream=b.stream)
    sim.init(*fields)
    with pytest.raises(pond.PondError):
        b.add(sim)
    b.close()
    sim.close()
