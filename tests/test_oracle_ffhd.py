"""Pins of the oracle's frozen-field hydrodynamics (Section 2.3.2, Eqs. 7-9): a fluid moving
along a frozen unit field b, with the source p div b in the field-aligned momentum equation.

Fixed independently of the FFHD code itself:
  * with b along a grid axis the system is 1-D Euler along that axis: the run must equal
    the oracle's HD run of the same Sod problem (same dt) in rho, m_par = m_axis and e;
  * at rest with uniform p in a curved field, the momentum flux p b and the source p div b
    must cancel, so nothing moves;
  * uniform v_par and p along an oblique uniform field stay uniform while the density is
    advected (the contact property of the flux), mass and energy are conserved;
  * reflecting walls with flow into them conserve mass; b never changes.
"""
import math

import numpy as np
import pytest

from oracle import Config, Solver
from paper_2607_19277_gb300 import workloads as W

OUT, PER, REF = "outflow", "periodic", "reflect"


def _ffhd_ic(prim_fn, bfield):
    def f(x, y, z):
        p = np.zeros((6,) + np.shape(x))
        rho, v, pr = prim_fn(x, y, z)
        p[0], p[1], p[2] = rho, v, pr
        b = bfield(x, y, z)
        p[3:6] = b
        return p
    return f


@pytest.mark.parametrize("axis", [0, 1])
def test_axis_field_equals_hd(axis):
    bc = [PER] * 6
    bc[2 * axis] = bc[2 * axis + 1] = OUT
    bb = [1, 1, 1]
    bb[axis] = 2
    hd = Solver(Config(physics="hd", limiter="minmod", flux="tvdlf", rk=2, base_blocks=tuple(bb), bc=tuple(bc)))
    hd.set_state(W.sod_axis(axis))
    ff = Solver(Config(physics="ffhd", limiter="minmod", flux="tvdlf", rk=2, base_blocks=tuple(bb), bc=tuple(bc)))

    def sod(x, y, z):
        p = W.sod_axis(axis)(x, y, z)
        return p[0], p[1 + axis], p[4]

    def bfield(x, y, z):
        b = np.zeros((3,) + np.shape(x))
        b[axis] = 1.0
        return b
    ff.set_state(_ffhd_ic(sod, bfield))
    for _ in range(6):
        hd.step(2e-3)
        ff.step(2e-3)
    _, _, ch = hd.get_state()
    _, _, cf = ff.get_state()
    for vf, vh in ((0, 0), (1, 1 + axis), (2, 4)):
        err = np.max(np.abs(cf[:, vf] - ch[:, vh])) / np.max(np.abs(ch[:, vh]))
        assert err < 1e-13, (vf, err)
    assert np.max(np.abs(ch[:, 1 + axis])) > 1e-2       # the problem moves


def _curved(x, y, z):
    th = 0.7 * np.sin(2 * math.pi * x) + 0.5 * np.cos(2 * math.pi * (y + z))
    b = np.zeros((3,) + np.shape(x))
    b[0] = np.cos(th) * np.cos(0.3 * th)
    b[1] = np.sin(th) * np.cos(0.3 * th)
    b[2] = np.sin(0.3 * th)
    return b


@pytest.mark.parametrize("rk", [2, 3])
def test_rest_in_curved_field_stays_at_rest(rk):
    s = Solver(Config(physics="ffhd", limiter="vanleer", flux="tvdlf", rk=rk, base_blocks=(2, 1, 1)))
    s.set_state(_ffhd_ic(lambda x, y, z: (1.3 + 0 * x, 0 * x, 0.7 + 0 * x), _curved))
    _, _, c0 = s.get_state()
    for _ in range(3):
        s.step(1e-2)
    _, _, c1 = s.get_state()
    assert np.max(np.abs(c1[:, 1])) < 1e-14          # no momentum appears
    assert np.max(np.abs(c1[:, [0, 2]] - c0[:, [0, 2]])) < 1e-14
    assert np.array_equal(c1[:, 3:], c0[:, 3:])       # the field is frozen


def test_uniform_flow_along_oblique_field_advects_density():
    b0 = np.array([1.0, 1.0, 0.5]) / 1.5

    def prim(x, y, z):
        rho = 1.0 + 0.3 * np.sin(2 * math.pi * (x + y))
        return rho, 0.8 + 0 * x, 1.1 + 0 * x

    def field(x, y, z):
        return np.broadcast_to(b0.reshape(3, *([1] * np.ndim(x))), (3,) + np.shape(x)).copy()
    s = Solver(Config(physics="ffhd", limiter="vanleer", flux="tvdlf", rk=3, base_blocks=(2, 2, 1)))
    s.set_state(_ffhd_ic(prim, field))
    s0 = s.conserved_sums()
    _, _, c0 = s.get_state()
    for _ in range(5):
        s.step()
    _, _, c1 = s.get_state()
    P, _ = s.phys.cons2prim(np.moveaxis(c1, 1, 0))
    assert np.max(np.abs(P[1] - 0.8)) < 1e-13 and np.max(np.abs(P[2] - 1.1)) < 1e-13
    assert np.max(np.abs(c1[:, 0] - c0[:, 0])) > 1e-3      # the density moved
    s1 = s.conserved_sums()
    assert abs(s1[0] - s0[0]) < 1e-14 * s0[0] and abs(s1[2] - s0[2]) < 1e-14 * s0[2]


def test_reflecting_walls_conserve_mass():
    s = Solver(Config(physics="ffhd", limiter="minmod", flux="tvdlf", rk=2, base_blocks=(1, 1, 1),
                      bc=(REF,) * 6))
    s.set_state(_ffhd_ic(lambda x, y, z: (1.0 + 0.2 * np.cos(3 * x), 0.5 + 0 * x, 1.0 + 0.1 * y), _curved))
    m0 = s.conserved_sums()[0]
    _, _, c0 = s.get_state()
    for _ in range(4):
        s.step()
    _, _, c1 = s.get_state()
    assert abs(s.conserved_sums()[0] - m0) < 1e-14 * m0
    assert np.array_equal(c1[:, 3:], c0[:, 3:])


def test_ffhd_requires_uniform_mesh():
    with pytest.raises(ValueError):
        Solver(Config(physics="ffhd", flux="tvdlf", max_level=2))
