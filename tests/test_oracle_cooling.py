"""Pins of the oracle's radiative-loss integration (Townsend 2009 exact integration, the
method Section 2.3.1 names for the sink -n_e n_H Lambda(T) of Eq. 4; code units
de/dt = -rho^2 Lambda(T), T = p / rho).

Fixed independently of the oracle's own formulas:
  * one power-law segment: dT/dt = -k T^a with k = (gamma - 1) rho Lambda_0 T_0^-a has the
    closed form T^(1-a)(t) = T^(1-a)(0) - (1 - a) k t (a != 1) and T(0) exp(-k t) (a = 1);
  * a many-node table: scipy's adaptive ODE integration of dT/dt with Lambda interpolated
    linearly in (ln T, ln Lambda) by this test;
  * the floor T_0, exact composition of two half steps, and the first-order drop in a
    tiny step resolved to the local cooling time;
  * the conserved update changes only e, by rho (T_new - T) / (gamma - 1);
  * a static uniform state through a full solver step (Strang halves compose exactly).
"""
import math

import numpy as np
import pytest

from oracle import Config, Solver
from oracle.cooling import Cooling
from oracle.physics import HD, MHD
from paper_2607_19277_gb300 import workloads as W

integrate = pytest.importorskip("scipy.integrate")


@pytest.mark.parametrize("a", [0.5, 1.0, -1.0, 2.5])
def test_single_power_law_closed_form(a):
    gamma, rho = 1.4, 2.5
    t0, t1 = 1.0, 4.0
    l0 = 0.3
    cool = Cooling([t0, t1], [l0, l0 * (t1 / t0) ** a], gamma)
    assert cool.alpha[0] == pytest.approx(a, rel=1e-14)
    k = (gamma - 1.0) * rho * l0 * t0 ** (-a)
    T = np.array([3.9, 3.0, 2.2, 1.5])
    for dt in (1e-3, 0.05, 0.2):
        got = cool.cool_temperature(rho, T, dt)
        if a == 1.0:
            want = T * np.exp(-k * dt)
        else:
            want = (T ** (1.0 - a) - (1.0 - a) * k * dt) ** (1.0 / (1.0 - a))
        want = np.maximum(want, t0)
        assert np.allclose(got, want, rtol=1e-13, atol=0), (a, dt, got, want)


def test_table_matches_adaptive_ode_integration():
    T, L = W.skew_normal_cooling(n=64)
    gamma, rho = 5.0 / 3.0, 1.7
    cool = Cooling(T, L, gamma)
    lnT, lnL = np.log(T), np.log(L)

    def lam(t):
        if t <= T[0]:
            return 0.0
        if t >= T[-1]:     # the last segment continues above the table
            s = (lnL[-1] - lnL[-2]) / (lnT[-1] - lnT[-2])
            return math.exp(lnL[-1] + s * (math.log(t) - lnT[-1]))
        return math.exp(np.interp(math.log(t), lnT, lnL))

    for t_start in (0.05, 0.3, 2.0, 50.0, 150.0):
        for dt in (1e-3, 0.1, 1.0):
            sol = integrate.solve_ivp(lambda _, y: [-(gamma - 1.0) * rho * lam(y[0])], (0.0, dt), [t_start],
                                      method="DOP853", rtol=1e-12, atol=1e-14)
            want = max(sol.y[0, -1], T[0])
            got = cool.cool_temperature(rho, np.array([t_start]), dt)[0]
            assert abs(got - want) <= 1e-10 * want, (t_start, dt, got, want)


def test_floor_composition_and_local_precision():
    T, L = W.skew_normal_cooling(n=32, peak=20.0)
    cool = Cooling(T, L, 5.0 / 3.0)
    # a very long step ends exactly on the floor; at or below the floor nothing changes
    assert np.all(cool.cool_temperature(1.0, np.array([0.5, 5.0, 80.0]), 1e9) == T[0])
    low = np.array([T[0], 0.5 * T[0]])
    assert np.array_equal(cool.cool_temperature(1.0, low, 10.0), low)
    # exact integration composes: two halves equal the whole step
    t = np.array([0.02, 0.2, 0.31, 1.0, 7.0, 60.0, 140.0])
    for dt in (1e-4, 1e-2, 0.3):
        half = cool.cool_temperature(1.2, cool.cool_temperature(1.2, t, 0.5 * dt), 0.5 * dt)
        full = cool.cool_temperature(1.2, t, dt)
        assert np.allclose(half, full, rtol=1e-12, atol=0), dt
    # first order in a tiny step, to the precision of the local cooling time: near the
    # peak 1/Lambda at the table's top exceeds the local scale by ~1e6
    lam = np.exp(np.interp(np.log(t), np.log(T), np.log(L)))
    top = t > T[-1]                                    # the last power law continues
    slope = np.log(L[-1] / L[-2]) / np.log(T[-1] / T[-2])
    lam[top] = L[-1] * (t[top] / T[-1]) ** slope
    dt = 1e-8 * t / ((2.0 / 3.0) * 1.2 * lam)          # dt / t_cool = 1e-8
    drop = (t - cool.cool_temperature(1.2, t, dt)) / t
    assert np.max(np.abs(drop / 1e-8 - 1.0)) < 1e-6


@pytest.mark.parametrize("phys", [HD(5.0 / 3.0), MHD(5.0 / 3.0)])
def test_conserved_update_changes_only_energy(phys):
    T, L = W.skew_normal_cooling(n=48)
    cool = Cooling(T, L, phys.gamma)
    rng = np.random.default_rng(3)
    n = 200
    P = np.zeros((phys.nvar, n))
    P[0] = rng.uniform(0.5, 2.0, n)
    P[1:4] = rng.normal(size=(3, n))
    P[4] = P[0] * np.exp(rng.uniform(np.log(0.02), np.log(40.0), n))
    if phys.nvar == 9:
        P[5:8] = rng.normal(size=(3, n))
        P[8] = rng.normal(size=n)
    U = phys.prim2cons(P)
    out = cool.apply(phys, U, 0.01)
    keep = [v for v in range(phys.nvar) if v != 4]
    assert np.array_equal(out[keep], U[keep])
    tn = cool.cool_temperature(P[0], P[4] / P[0], 0.01)
    de = P[0] * (P[4] / P[0] - tn) / (phys.gamma - 1.0)
    assert np.max(np.abs(out[4] - (U[4] - de)) / np.abs(U[4])) < 1e-14
    assert np.all(out[4] <= U[4])


@pytest.mark.parametrize("physics", ["hd", "mhd"])
def test_static_state_step_equals_exact_cooling(physics):
    T, L = W.skew_normal_cooling(n=64)
    prim = [1.3, 0.0, 0.0, 0.0, 1.3 * 0.8] + ([0.4, -0.2, 0.3, 0.0] if physics == "mhd" else [])
    s = Solver(Config(physics=physics, flux="hll", limiter="vanleer", rk=3, base_blocks=(1, 1, 1),
                      cooling=(T, L)))
    s.set_state(W.uniform_state(prim))
    dt = 0.02
    s.step(dt, ch=1.0)
    _, _, c = s.get_state()
    ph = s.phys
    p, _ = ph.cons2prim(c[0, :ph.nvar].reshape(ph.nvar, -1))
    tn = Cooling(T, L, 5.0 / 3.0).cool_temperature(1.3, np.array([0.8]), dt)[0]
    assert np.allclose(p[4] / p[0], tn, rtol=1e-13)
    assert tn < 0.8 * (1 - 1e-4)          # the losses are not negligible at this dt


def test_power_law_near_one_is_continuous():
    """alpha within 1e-10 of 1: the expm1 / log1p forms must reproduce the exponential decay
    of the alpha = 1 law (a naive (x^e - 1)/e loses about 1e-6 here)."""
    gamma, rho, t0, t1, l0 = 1.4, 2.5, 1.0, 4.0, 0.3
    k = (gamma - 1.0) * rho * l0 / t0
    for a in (1.0 - 1e-10, 1.0 + 1e-10):
        cool = Cooling([t0, t1], [l0, l0 * (t1 / t0) ** a], gamma)
        T = np.array([3.9, 2.0])
        got = cool.cool_temperature(rho, T, 0.1)
        assert np.allclose(got, T * np.exp(-k * 0.1), rtol=1e-8)
