"""The bound behind the estimator's FP32 screen for refinement decisions.

For a regrid the library evaluates the Loehner estimate of every cell in FP32 first and
runs the exact FP64 evaluation only for blocks whose FP32 maximum lies within a margin of
a threshold. The margin is four times sum_i |w_i| (8 u / eps + 32 u), u = 2^-24: the FP32
value of one variable's estimate must stay within 8 u / eps + 32 u of the exact value for
stencils inside the screen's range (magnitudes between 1e-10 and 1e18). This checks that
bound on random stencils with numpy's IEEE FP32 arithmetic, in the kernel's order of
operations: smooth (nearly linear) stencils, nearly cancelling ones around a large offset,
and arbitrary ones, over sixteen orders of magnitude."""
import numpy as np


def _estimate(a, o, m, eps, dtype):
    a, o, m = (x.astype(dtype) for x in (a, o, m))
    e = dtype(eps)
    two = dtype(2)
    num = np.zeros(a.shape[0], dtype)
    den = np.zeros(a.shape[0], dtype)
    for d in range(3):
        tt = (a[:, d] - two * o[:, d]) + m[:, d]
        sm = (np.abs(a[:, d]) + two * np.abs(o[:, d])) + np.abs(m[:, d])
        q = (np.abs(a[:, d] - o[:, d]) + np.abs(o[:, d] - m[:, d])) + e * sm
        num = num + tt * tt
        den = den + q * q
    safe = np.where(den > 0, den, dtype(1))
    return np.where(den > 0, np.sqrt(num / safe), dtype(0)).astype(np.float64)


def test_fp32_estimate_within_screen_bound():
    rng = np.random.default_rng(20260905)
    eps, u = 0.01, 2.0 ** -24
    bound = 8 * u / eps + 32 * u
    n = 300000
    scale = 10.0 ** rng.uniform(-8, 8, size=(n, 1))
    kind = rng.integers(0, 3, size=n)[:, None]
    o = rng.uniform(-1, 1, size=(n, 3))
    a = np.where(kind == 0, o + 1e-6 * rng.standard_normal((n, 3)), rng.uniform(-1, 1, size=(n, 3)))
    m = np.where(kind == 0, o - 1e-6 * rng.standard_normal((n, 3)), rng.uniform(-1, 1, size=(n, 3)))
    o = np.where(kind == 2, 1 + 1e-7 * rng.standard_normal((n, 3)), o)
    # the stored values are FP32 (the FP32 stencil's pools)
    a, o, m = ((x * scale).astype(np.float32) for x in (a, o, m))
    exact = _estimate(a, o, m, eps, np.float64)
    fp32 = _estimate(a, o, m, eps, np.float32)
    assert np.all(exact <= 1.0 + 1e-12)               # the estimate never exceeds 1
    err = np.abs(fp32 - exact)
    assert err.max() < bound, (err.max(), bound)
    # a plausible mistake in the screen's arithmetic (eps dropped from the denominator)
    # leaves cancelling stencils unbounded: the check would catch it
    bad = _estimate(a, o, m, 0.0, np.float32)
    assert np.abs(bad - _estimate(a, o, m, 0.0, np.float64)).max() > bound
