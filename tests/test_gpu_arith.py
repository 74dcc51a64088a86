"""The step kernels' own FP64 arithmetic helpers against CUDA's correctly
rounded operations, on the GPU.

The van Leer limiter of the FP64 path forms x y / (x + y) as x y times a
reciprocal from the hardware approximation refined by one Newton-Raphson step
(FMA form of Newton's iteration, Markstein 1990).  One step squares the
relative error of the approximation (about 2^-20), so the reciprocal is good
to about 2^-40; the stated bound checked here is 2^-39 relative over the
normal range 2^-1021 <= |y| <= 2^1021.  Outside it (subnormal y, or 1/y
subnormal) the approximation flushes and the result is not finite, or zero;
the limiter never meets such a denominator: its
denominator x + y is a sum of two same-signed differences of node values, and
a product x y below 2^-1042 (high word zero) already counts as no slope.
"""
import numpy as np
import pytest

from paper_2302_00310_gb300 import pond

pytestmark = pytest.mark.gpu
N = 1 << 20
# one Newton step squares the approximation's relative error (measured below
# 2^-19.9 over these operands), so the reciprocal is good to 2^-39 (measured
# 9.7e-13 = 2^-39.9 on GB300)
RCP_BOUND = 2.0 ** -39


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    pond.lib(build=True)
    return t


def _random_doubles(rng, n, emin, emax):
    """Random signs, mantissas uniform in [1, 2), exponents uniform in [emin, emax]."""
    m = rng.uniform(1.0, 2.0, n)
    e = rng.integers(emin, emax + 1, n)
    s = rng.choice([-1.0, 1.0], n)
    return s * np.ldexp(m, e)


def test_reciprocal_within_its_bound_over_the_normal_range(torch):
    rng = np.random.default_rng(2024)
    y = _random_doubles(rng, N, -1021, 1020)
    y[:4] = [1.0, -1.0, 2.0 ** -1021, -(2.0 ** 1020)]
    yd = torch.from_numpy(y).cuda()
    r, ref = torch.empty_like(yd), torch.empty_like(yd)
    pond.pond_check_reciprocal(yd, r, ref)
    r, ref = r.cpu().numpy(), ref.cpu().numpy()
    assert np.all(np.isfinite(r)) and np.all(np.sign(r) == np.sign(y))
    assert np.array_equal(ref, 1.0 / y)  # CUDA's __drcp_rn is the correctly rounded reciprocal
    err = np.max(np.abs(r - ref) / np.abs(ref))
    assert err <= RCP_BOUND, err


def test_reciprocal_outside_the_normal_range_flushes(torch):
    """Subnormal y: the .ftz approximation reads it as zero, and the Newton
    step then meets inf * 0 (NaN); 1/y subnormal: flushed to zero.  Neither
    input reaches the limiter (see the module docstring)."""
    y = np.array([2.0 ** -1030, -(2.0 ** -1060), 2.0 ** 1023, -(2.0 ** 1023)])
    yd = torch.from_numpy(y).cuda()
    r, ref = torch.empty_like(yd), torch.empty_like(yd)
    pond.pond_check_reciprocal(yd, r, ref)
    r = r.cpu().numpy()
    assert not np.isfinite(r[0]) and not np.isfinite(r[1])
    assert r[2] == 0.0 and r[3] == 0.0


def test_vanleer_limiter_against_correctly_rounded_division(torch):
    rng = np.random.default_rng(7)
    x = _random_doubles(rng, N, -300, 300)
    # pairs of similar magnitude (the common case: neighbouring differences)
    # and pairs far apart; signs independent, so half the pairs have no slope
    y = np.where(rng.random(N) < 0.5, x * rng.uniform(-3.0, 3.0, N), _random_doubles(rng, N, -300, 300))
    # subnormal operands and products that underflow
    x[:6] = [1e-310, -1e-310, 2e-310, 5e-320, 1e-200, 3.0]
    y[:6] = [1e-310, -3e-311, 2e-10, 5e-320, 1e-200, 0.0]
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    l, ref = torch.empty_like(xd), torch.empty_like(xd)
    pond.pond_check_vanleer(xd, yd, l, ref)
    l, ref = l.cpu().numpy(), ref.cpu().numpy()
    p = x * y
    # no slope where x y <= 0, exactly, on both sides
    assert np.all(l[p <= 0] == 0.0) and np.all(ref[p <= 0] == 0.0)
    # elsewhere the reciprocal's bound, plus an absolute floor far below any
    # physical slope for products under 2^-1042 (the kernel counts them as 0)
    err = np.abs(l - ref)
    assert np.all(err <= RCP_BOUND * np.abs(ref) + 2.0 ** -1000), np.max(err / np.maximum(np.abs(ref), 1e-300))
    assert np.all(np.isfinite(l))
