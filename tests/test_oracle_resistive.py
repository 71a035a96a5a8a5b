"""Pins of the oracle's resistive MHD terms (Section 2.3.3: -curl(eta J) in the induction
equation, div(B x eta J) in the energy equation, added as sources with a compact stencil).

  * eta = 0 is ideal MHD bit for bit                                   -> the switch
  * a field mode B_perp = eps sin(2 pi x_d) at rest decays as
    exp(-eta (2 pi)^2 t), at second order, for three axis / component
    pairings (each uses a different component of J and of lap B)         -> lap B, J, indices
  * the total energy is conserved to truncation order: the Ohmic heating
    eta J^2 returns what eta B.lap B takes from the magnetic energy
    (a dropped or sign-flipped term leaves a change of order 1), for
    every component of J                                                 -> energy source
  * mass, momentum and B are conserved to round-off on a periodic mesh  -> source form of B
  * the diffusive time-step bound scales as dx^2                        -> dt
"""
import math

import numpy as np
import pytest

from oracle import Config, Solver
from paper_2607_19277_gb300 import workloads as W


def _mode_state(axis, comp, eps):
    def ic(x, y, z):
        q = (np.asarray(x), np.asarray(y), np.asarray(z))[axis]
        P = np.zeros((9, q.size))
        P[0] = 1.0
        P[4] = 1.0
        P[5 + comp] = eps * np.sin(2 * math.pi * q)
        return P
    return ic


def _thin(n, axis, **kw):
    """n cells along `axis` on [0, 1], one block across with cells twice as wide (an axis
    mixed up in the stencil then takes the wrong spacing)."""
    bb = [1, 1, 1]
    bb[axis] = n // 16
    xmax = [32.0 / n] * 3
    xmax[axis] = 1.0
    return Solver(Config(physics="mhd", limiter="vanleer", flux="hll", rk=2, base_blocks=tuple(bb),
                         xmax=tuple(xmax), **kw))


def _decay_error(n, axis, comp, eta=0.05, eps=1e-3, decay=0.15):
    """Mean |B_comp - exact| / eps after the mode decayed by exp(-decay)."""
    s = _thin(n, axis, eta=eta)
    s.set_state(_mode_state(axis, comp, eps))
    tend = decay / (eta * (2 * math.pi) ** 2)
    t = 0.0
    while t < tend - 1e-14:
        t += s.step(min(s.cfl_dt(), tend - t))
    err = 0.0
    cnt = 0
    for k, blk in s.leaves.items():
        q = s.cell_centres(k)[axis]
        b = blk[5 + comp, 2:18, 2:18, 2:18].ravel()
        err += np.abs(b - eps * math.exp(-decay) * np.sin(2 * math.pi * q)).sum()
        cnt += b.size
    return err / cnt / eps


@pytest.mark.parametrize("axis,comp", [(0, 1), (1, 2), (2, 0)])
def test_field_mode_decays_at_the_resistive_rate_second_order(axis, comp):
    e = [_decay_error(n, axis, comp) for n in (16, 32)]
    assert math.log2(e[0] / e[1]) >= 1.8, e
    assert e[1] < 1.5e-3, e


def test_eta_zero_is_ideal_mhd():
    res = []
    for kw in ({}, {"eta": 0.0}):
        s = Solver(Config(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 1, 1), **kw))
        s.set_state(W.random_smooth(9, 51, "mhd"))
        for _ in range(2):
            s.step()
        res.append(s.get_state()[2])
    assert np.array_equal(res[0], res[1])


def _energy_budget(n, axis, comp, eta=0.05, eps=0.05):
    s = _thin(n, axis, eta=eta)
    s.set_state(_mode_state(axis, comp, eps))

    def emag():
        return sum(0.5 * (blk[5:8, 2:18, 2:18, 2:18] ** 2).sum() for blk in s.leaves.values())
    e0, m0 = s.conserved_sums()[4], emag()
    for _ in range(8):
        s.step()
    vol = np.prod(s.dx(1))
    return (s.conserved_sums()[4] - e0) / ((emag() - m0) * vol)


@pytest.mark.parametrize("axis,comp", [(0, 1), (1, 0), (1, 2), (2, 1), (2, 0), (0, 2)])
def test_ohmic_heating_balances_the_magnetic_energy_loss(axis, comp):
    """Each pairing of a field component with a direction it varies along exercises one of
    the six derivative terms of J = curl B."""
    r = [abs(_energy_budget(n, axis, comp)) for n in (16, 32)]
    # |change of total energy| / |change of magnetic energy| -> 0 as (k dx)^2 / 4
    assert r[0] < 0.05 and r[1] < 0.015, r
    assert math.log2(r[0] / r[1]) >= 1.8, r


def test_resistive_run_conserves_mass_momentum_and_b():
    s = Solver(Config(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 2, 1), eta=0.02))
    s.set_state(W.random_smooth(9, 52, "mhd"))
    s0 = s.conserved_sums()
    for _ in range(3):
        s.step()
    s1 = s.conserved_sums()
    keep = [0, 1, 2, 3, 5, 6, 7]
    assert np.max(np.abs(s1[keep] - s0[keep])) <= 1e-13 * np.abs(s0[keep]).max()


def test_diffusive_bound_scales_with_dx_squared():
    dts = []
    for n in (16, 32):
        s = _thin(n, 0, eta=10.0)
        s.set_state(_mode_state(0, 1, 1e-3))
        dts.append(s.cfl_dt())
    assert dts[0] / dts[1] == pytest.approx(4.0, rel=1e-12)
