"""GPU parity of frozen-field hydrodynamics with hyperbolic thermal conduction (Section
2.3.2, Eqs. 9-10) with the FP64 oracle: flow along a curved field with a heat flux (FP64 and
FP32, both limiters), reflecting and outflow walls, radiative losses together with
conduction, the decay polynomial of a uniform heat flux, conservation, and the batched path."""
import math

import numpy as np
import pytest

from oracle import Config, Solver
from paper_2607_19277_gb300 import agile, workloads as W
from parity_util import TOL_FP32, TOL_FP64, rel_l1, run_both

pytestmark = pytest.mark.gpu
OUT, PER, REF = "outflow", "periodic", "reflect"
KAPPA0 = 0.05


def _field(x, y, z):
    th = 0.7 * np.sin(2 * math.pi * x) + 0.5 * np.cos(2 * math.pi * (y + z))
    b = np.zeros((3,) + np.shape(x))
    b[0] = np.cos(th) * np.cos(0.3 * th)
    b[1] = np.sin(th) * np.cos(0.3 * th)
    b[2] = np.sin(0.3 * th)
    return b


def _flow(x, y, z):
    p = np.zeros((7,) + np.shape(x))
    p[0] = 1.0 + 0.3 * np.sin(2 * math.pi * (x + 2 * y)) * np.cos(2 * math.pi * z)
    p[1] = 0.4 * np.cos(2 * math.pi * (x - y))
    p[2] = 1.0 + 0.4 * np.sin(2 * math.pi * (y + z)) * np.cos(2 * math.pi * x)
    p[3] = 0.05 * np.sin(2 * math.pi * (x + y - z))
    p[4:7] = _field(x, y, z)
    return p


def _rel(g, r):
    return rel_l1(g, r)[:4]       # rho, m_par, e, q_par (the frozen field is exact)


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, TOL_FP32)])
@pytest.mark.parametrize("limiter", ["minmod", "vanleer"])
def test_conduction_along_curved_field(rb, tol, limiter):
    spec = dict(physics="ffhd_htc", htc_kappa0=KAPPA0, limiter=limiter, flux="tvdlf", rk=3,
                base_blocks=(2, 2, 2))
    m, o, g, r, lev, _ = run_both(spec, _flow, 4, real_bytes=rb)
    assert _rel(g, r).max() < tol, _rel(g, r)
    assert np.max(np.abs(r[:, 3])) > 1e-3          # the heat flux is active
    m.close()


@pytest.mark.parametrize("bc", [(REF,) * 6, (OUT, OUT, PER, PER, REF, REF)])
def test_walls_fp64(bc):
    spec = dict(physics="ffhd_htc", htc_kappa0=KAPPA0, limiter="minmod", flux="tvdlf", rk=2,
                base_blocks=(2, 1, 1), bc=bc)
    m, o, g, r, lev, _ = run_both(spec, _flow, 4)
    assert _rel(g, r).max() < TOL_FP64
    m.close()


def test_losses_and_conduction_fp64():
    tab = W.skew_normal_cooling(n=128, peak=20.0)
    spec = dict(physics="ffhd_htc", htc_kappa0=KAPPA0, limiter="vanleer", flux="tvdlf", rk=3,
                base_blocks=(2, 2, 1))
    m = agile.Mesh(agile.make_config(real_bytes=8, **spec))
    m.set_cooling(*tab)
    m.set_state(_flow)
    o = Solver(Config(cooling=tab, **spec))
    o.set_state(_flow)
    for _ in range(3):
        dt = m.cfl_dt()
        m.step(dt)
        o.step(dt)
    _, _, g = m.get_state()
    _, _, r = o.get_state()
    m.close()
    assert _rel(g, r).max() < TOL_FP64


@pytest.mark.parametrize("rk,factor", [(2, 1 - 0.25 + 0.25 ** 2 / 2),
                                       (3, 1 - 0.25 + 0.25 ** 2 / 2 - 0.25 ** 3 / 6)])
def test_uniform_heat_flux_decay(rk, factor):
    m = agile.Mesh(agile.make_config(physics="ffhd_htc", htc_kappa0=0.3, limiter="vanleer", flux="tvdlf", rk=rk,
                                     base_blocks=(1, 1, 1)))
    q0 = 0.7

    def ic(x, y, z):
        p = np.zeros((7,) + np.shape(x))
        p[0], p[2], p[3] = 1.2, 0.9, q0
        p[4], p[5], p[6] = 0.8, 0.6, 0.0
        return p
    m.set_state(ic)
    for n in range(1, 4):
        m.step(1e-3)
        _, _, c = m.get_state()
        assert np.max(np.abs(c[:, 3] - q0 * factor ** n)) < 1e-14
    m.close()


def test_conservation_fp32():
    m = agile.Mesh(agile.make_config(physics="ffhd_htc", htc_kappa0=KAPPA0, limiter="vanleer", flux="tvdlf",
                                     rk=3, real_bytes=4, base_blocks=(2, 2, 2)))
    m.set_state(_flow)
    s0 = m.conserved_sums()
    for _ in range(5):
        m.step(m.cfl_dt())
    s1 = m.conserved_sums()
    m.close()
    for v in (0, 2):
        assert abs(s1[v] - s0[v]) <= 1e-6 * abs(s0[v])


def test_batch_equals_alone():
    cfgs = [agile.make_config(physics="ffhd_htc", htc_kappa0=KAPPA0, limiter="vanleer", flux="tvdlf", rk=3,
                              real_bytes=4, base_blocks=(n, n, n)) for n in (2, 3)]
    b = agile.Batch(cfgs)
    alone = []
    for i, c in enumerate(cfgs):
        b.set_state(i, _flow)
        m = agile.Mesh(c)
        m.set_state(_flow)
        alone.append(m)
    for _ in range(3):
        b.step()
        for m in alone:
            m.step(0.0)
    for i, m in enumerate(alone):
        assert np.array_equal(b.get_state(i)[2], m.get_state()[2]), i
        m.close()
    b.close()
