"""Pins of the oracle's hyperbolic thermal conduction in frozen-field hydrodynamics
(Section 2.3.2, Eqs. 9-10): q_par relaxes towards kappa0 T^(5/2) b.grad T over tau = 4 dt
and carries energy along the field through the flux -q_par b.

Fixed independently of the HTC code itself:
  * uniform state, uniform q_par: the target vanishes, so q_par decays by the stability
    polynomial of the SSPRK scheme at z = dt / tau = 1/4 per step (1 - z + z^2/2 for
    SSPRK2, 1 - z + z^2/2 - z^3/6 for SSPRK3), while rho, m_par and e stay put;
  * kappa0 = 0 and q_par = 0: the run is the plain FFHD run;
  * periodic domain: mass and energy are conserved to round-off with conduction on;
  * a hot spot on a straight field cools faster than without conduction and heats its
    neighbours along the field (heat flows down the temperature gradient), and not across;
  * the target on a quadratic temperature field equals kappa0 T^(5/2) b.grad T with the
    analytic gradient (central differences are exact for quadratics), for an oblique b.
"""
import math

import numpy as np
import pytest

from oracle import Config, Solver
from oracle.physics import FFHDHTC

OUT, PER = "outflow", "periodic"


def _ic(prim_fn, bfield, q_fn=None):
    def f(x, y, z):
        p = np.zeros((7,) + np.shape(x))
        rho, v, pr = prim_fn(x, y, z)
        p[0], p[1], p[2] = rho, v, pr
        p[3] = 0.0 if q_fn is None else q_fn(x, y, z)
        p[4:7] = bfield(x, y, z)
        return p
    return f


def _uniform_b(b):
    b = np.asarray(b, float) / np.linalg.norm(b)

    def f(x, y, z):
        return np.broadcast_to(b.reshape(3, *([1] * np.ndim(x))), (3,) + np.shape(x)).copy()
    return f


@pytest.mark.parametrize("rk,factor", [(2, 1 - 0.25 + 0.25 ** 2 / 2),
                                       (3, 1 - 0.25 + 0.25 ** 2 / 2 - 0.25 ** 3 / 6)])
def test_uniform_heat_flux_decays_by_the_rk_polynomial(rk, factor):
    s = Solver(Config(physics="ffhd_htc", htc_kappa0=0.3, limiter="vanleer", flux="tvdlf", rk=rk,
                      base_blocks=(1, 1, 1)))
    q0 = 0.7
    s.set_state(_ic(lambda x, y, z: (1.2 + 0 * x, 0 * x, 0.9 + 0 * x), _uniform_b([1.0, 0.5, 0.25]),
                    lambda x, y, z: q0 + 0 * x))
    _, _, c0 = s.get_state()
    for n in range(1, 4):
        s.step(1e-3 * n)              # the factor does not depend on dt
        _, _, c = s.get_state()
        assert np.max(np.abs(c[:, 3] - q0 * factor ** n)) < 1e-14
    assert np.max(np.abs(c[:, [0, 1, 2]] - c0[:, [0, 1, 2]])) < 1e-13
    assert np.array_equal(c[:, 4:], c0[:, 4:])


def _curved(x, y, z):
    th = 0.7 * np.sin(2 * math.pi * x) + 0.5 * np.cos(2 * math.pi * (y + z))
    b = np.zeros((3,) + np.shape(x))
    b[0] = np.cos(th) * np.cos(0.3 * th)
    b[1] = np.sin(th) * np.cos(0.3 * th)
    b[2] = np.sin(0.3 * th)
    return b


def _smooth(x, y, z):
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * (x + 2 * y))
    v = 0.3 * np.cos(2 * math.pi * z)
    p = 1.0 + 0.3 * np.cos(2 * math.pi * (x - y + z))
    return rho, v, p


def test_zero_conductivity_reduces_to_ffhd():
    cfg = dict(limiter="vanleer", flux="tvdlf", rk=3, base_blocks=(2, 1, 1))
    a = Solver(Config(physics="ffhd", **cfg))
    b = Solver(Config(physics="ffhd_htc", htc_kappa0=0.0, **cfg))

    def ffhd_ic(x, y, z):
        p = np.zeros((6,) + np.shape(x))
        p[0], p[1], p[2] = _smooth(x, y, z)
        p[3:6] = _curved(x, y, z)
        return p
    a.set_state(ffhd_ic)
    b.set_state(_ic(_smooth, _curved))
    for _ in range(3):
        dt = a.cfl_dt()
        assert dt == b.cfl_dt()
        a.step(dt)
        b.step(dt)
    _, _, ca = a.get_state()
    _, _, cb = b.get_state()
    assert np.array_equal(ca[:, :3], cb[:, :3])
    assert np.all(cb[:, 3] == 0.0)


def test_periodic_conduction_conserves_mass_and_energy():
    s = Solver(Config(physics="ffhd_htc", htc_kappa0=0.05, limiter="vanleer", flux="tvdlf", rk=2,
                      base_blocks=(2, 1, 1)))
    s.set_state(_ic(_smooth, _curved, lambda x, y, z: 0.05 * np.sin(2 * math.pi * y)))
    s0 = s.conserved_sums()
    for _ in range(4):
        s.step()
    s1 = s.conserved_sums()
    assert abs(s1[0] - s0[0]) < 1e-14 * s0[0]
    assert abs(s1[2] - s0[2]) < 1e-14 * s0[2]
    _, _, c = s.get_state()
    assert np.max(np.abs(c[:, 3])) > 1e-3        # conduction is active


def _hot_spot_run(kappa0, steps=6):
    s = Solver(Config(physics="ffhd_htc", htc_kappa0=kappa0, limiter="minmod", flux="tvdlf", rk=2,
                      base_blocks=(2, 1, 1), bc=(PER,) * 6))

    def prim(x, y, z):
        r2 = ((x - 0.5) / 0.08) ** 2 + ((y - 0.5) / 0.08) ** 2 + ((z - 0.5) / 0.08) ** 2
        return 1.0 + 0 * x, 0 * x, 1.0 + 2.0 * np.exp(-r2)
    s.set_state(_ic(prim, _uniform_b([1.0, 0.0, 0.0])))
    for _ in range(steps):
        s.step(2e-4)
    lev, ijk, c = s.get_state()
    P, _ = s.phys.cons2prim(np.moveaxis(c, 1, 0))
    T = P[2] / P[0]                                   # (block, z, y, x)
    return T, ijk


def test_hot_spot_cools_along_the_field():
    T1, ijk = _hot_spot_run(0.02)
    T0, _ = _hot_spot_run(0.0)
    # global cell indices of the 2x1x1 block mesh (32 x 16 x 16 cells)
    full1 = np.zeros((16, 16, 32))
    full0 = np.zeros((16, 16, 32))
    for b, (i, j, k) in enumerate(ijk.tolist()):
        full1[:, :, 16 * i:16 * i + 16] = T1[b]
        full0[:, :, 16 * i:16 * i + 16] = T0[b]
    zc, yc, xc = 8, 8, 16                             # cell centred nearest (0.5, 0.5, 0.5)
    assert full1[zc, yc, xc] < full0[zc, yc, xc] - 1e-4          # the spot cools faster
    assert full1[zc, yc, xc + 4] > full0[zc, yc, xc + 4] + 1e-6  # heat arrives along b
    # across the field (y) conduction adds nothing beyond rounding-level coupling
    assert abs(full1[zc, yc + 4, xc] - full0[zc, yc + 4, xc]) < 0.1 * abs(
        full1[zc, yc, xc + 4] - full0[zc, yc, xc + 4])


def test_target_on_quadratic_temperature_matches_analytic_gradient():
    ph = FFHDHTC(5.0 / 3.0, kappa0=0.7)
    dx = (0.1, 0.2, 0.05)
    n = np.arange(20) - 2 + 0.5
    Z, Y, X = np.meshgrid(n * dx[2], n * dx[1], n * dx[0], indexing="ij")
    T = 1.0 + 0.3 * X - 0.2 * Y + 0.5 * Z + 0.4 * X * X + 0.1 * Y * Z - 0.3 * Z * Z
    rho = 1.0 + 0.1 * X
    b = np.array([0.6, -0.48, 0.64])
    P = np.zeros((7, 20, 20, 20))
    P[0] = rho
    P[2] = T * rho
    P[4], P[5], P[6] = b[0], b[1], b[2]
    g = ph.htc_target(P, dx)
    i = slice(2, 18)
    gx = 0.3 + 0.8 * X
    gy = -0.2 + 0.1 * Z
    gz = 0.5 + 0.1 * Y - 0.6 * Z
    Ti = T[i, i, i]
    ref = 0.7 * Ti ** 2.5 * (b[0] * gx + b[1] * gy + b[2] * gz)[i, i, i]
    assert np.max(np.abs(g - ref)) < 1e-12 * np.max(np.abs(ref))
