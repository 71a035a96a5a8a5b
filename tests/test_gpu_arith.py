"""The FP64 stencil forms every quotient as a * r, r the hardware reciprocal estimate of s
refined by one third-order Newton-Raphson step (r (1 + e + e^2), e = 1 - s r). Checked on the
device against the IEEE quotient: within one unit in the last place over divisors and
dividends spread across the FP64 exponent range, and over the ranges the stencil divides by
(densities, slope sums, speed intervals)."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import agile

pytestmark = pytest.mark.gpu


def _wide(rng, n, lo, hi):
    m = 1.0 + rng.random(n)
    e = rng.integers(lo, hi, n)
    return np.ldexp(m, e) * rng.choice([-1.0, 1.0], n)


def test_quotient_within_one_ulp_across_exponent_range():
    rng = np.random.default_rng(7)
    n = 1 << 22
    s = _wide(rng, n, -1000, 1000)
    q = _wide(rng, n, -900, 900)                         # keep a / s a normal number
    a = q * s
    ok = np.isfinite(a) & (np.abs(a) >= np.finfo(np.float64).tiny)
    mu, mr = agile.check_rcp64(s[ok], a[ok])
    assert mu <= 1.0, mu
    assert mr <= 2.0 ** -52, mr


def test_quotient_within_one_ulp_on_stencil_ranges():
    rng = np.random.default_rng(8)
    n = 1 << 20
    # densities and pressures over ten decades, slope sums of either sign, mantissas near
    # powers of two (where the last place changes size)
    s = np.concatenate([10.0 ** rng.uniform(-5, 5, n), rng.normal(0, 1e-3, n),
                        np.ldexp(1.0 - rng.random(n) * 1e-15, rng.integers(-40, 40, n))])
    s[s == 0.0] = 1.0
    a = np.concatenate([rng.normal(0, 1, n), rng.normal(0, 1e-6, n), 1.0 + rng.random(n)])
    mu, mr = agile.check_rcp64(s, a)
    assert mu <= 1.0, mu
    assert mr <= 2.0 ** -52, mr
