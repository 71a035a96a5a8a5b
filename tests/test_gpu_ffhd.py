"""GPU parity of frozen-field hydrodynamics (Section 2.3.2) with the FP64 oracle: flow along
a curved frozen field (FP64 and FP32), Sod along an axis-aligned field, rest in a curved
field, reflecting walls, radiative losses, and the batched path."""
import math

import numpy as np
import pytest

from oracle import Config, Solver
from paper_2607_19277_gb300 import agile, workloads as W
from parity_util import TOL_FP32, TOL_FP64, rel_l1, run_both

pytestmark = pytest.mark.gpu
OUT, PER, REF = "outflow", "periodic", "reflect"


def _field(x, y, z):
    th = 0.7 * np.sin(2 * math.pi * x) + 0.5 * np.cos(2 * math.pi * (y + z))
    b = np.zeros((3,) + np.shape(x))
    b[0] = np.cos(th) * np.cos(0.3 * th)
    b[1] = np.sin(th) * np.cos(0.3 * th)
    b[2] = np.sin(0.3 * th)
    return b


def _flow(x, y, z):
    p = np.zeros((6,) + np.shape(x))
    p[0] = 1.0 + 0.3 * np.sin(2 * math.pi * (x + 2 * y)) * np.cos(2 * math.pi * z)
    p[1] = 0.4 * np.cos(2 * math.pi * (x - y))
    p[2] = 1.0 + 0.2 * np.sin(2 * math.pi * (y + z))
    p[3:6] = _field(x, y, z)
    return p


def _rel(g, r):
    return rel_l1(g, r)[:3]       # the frozen field is compared separately


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, TOL_FP32)])
def test_flow_along_curved_field(rb, tol):
    spec = dict(physics="ffhd", limiter="vanleer", flux="tvdlf", rk=3, base_blocks=(2, 2, 2))
    m, o, g, r, lev, _ = run_both(spec, _flow, 4, real_bytes=rb)
    assert _rel(g, r).max() < tol
    # the field is frozen: what the initial condition gave, in the stencil precision
    if rb == 8:
        assert np.array_equal(g[:, 3:], r[:, 3:])
    else:
        assert np.array_equal(g[:, 3:], r[:, 3:].astype(np.float32).astype(np.float64))
    m.close()


def test_sod_along_axis_field_fp64():
    spec = dict(physics="ffhd", limiter="minmod", flux="tvdlf", rk=2, base_blocks=(4, 1, 1),
                bc=(OUT, OUT, PER, PER, PER, PER))

    def ic(x, y, z):
        s = W.sod_x(x, y, z)
        p = np.zeros((6,) + np.shape(x))
        p[0], p[1], p[2], p[3] = s[0], s[1], s[4], 1.0
        return p
    m, o, g, r, lev, _ = run_both(spec, ic, 10)
    assert _rel(g, r).max() < TOL_FP64
    m.close()


@pytest.mark.parametrize("rb,tol", [(8, 1e-14), (4, 1e-6)])
def test_rest_in_curved_field(rb, tol):
    m = agile.Mesh(agile.make_config(physics="ffhd", limiter="vanleer", flux="tvdlf", rk=3, real_bytes=rb,
                                     base_blocks=(2, 1, 1)))

    def ic(x, y, z):
        p = np.zeros((6,) + np.shape(x))
        p[0], p[2] = 1.3, 0.7
        p[3:6] = _field(x, y, z)
        return p
    m.set_state(ic)
    _, _, c0 = m.get_state()
    for _ in range(3):
        m.step(1e-2)
    _, _, c1 = m.get_state()
    m.close()
    assert np.max(np.abs(c1[:, 1])) < tol
    assert np.max(np.abs(c1[:, [0, 2]] - c0[:, [0, 2]])) < tol
    assert np.array_equal(c1[:, 3:], c0[:, 3:])


def test_reflecting_walls_fp64():
    spec = dict(physics="ffhd", limiter="minmod", flux="tvdlf", rk=2, base_blocks=(2, 1, 1), bc=(REF,) * 6)
    m, o, g, r, lev, _ = run_both(spec, _flow, 4)
    assert _rel(g, r).max() < TOL_FP64
    s = m.conserved_sums()
    m.close()
    assert np.isfinite(s).all()


def test_losses_fp64():
    tab = W.skew_normal_cooling(n=128, peak=20.0)
    spec = dict(physics="ffhd", limiter="vanleer", flux="tvdlf", rk=3, base_blocks=(2, 2, 1))
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


def test_batch_equals_alone():
    cfgs = [agile.make_config(physics="ffhd", limiter="vanleer", flux="tvdlf", rk=3, real_bytes=4,
                              base_blocks=(n, n, n)) for n in (2, 3)]
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
