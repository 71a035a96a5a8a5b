"""Pins of the oracle's approximate Synge-gas EOS for SRHD (Section 2.3.4, Eq. 22 and the
Mathews approximation the paper uses instead of the Bessel functions).

What fixes the EOS independently of the oracle's own formulas:
  * the Bessel-function definition h = K3(1/theta) / K2(1/theta) (scipy), which the
    approximation must follow within 2.1% at every temperature and exactly in both limits;
  * thermodynamics: along an isentrope dh = dp / rho, so with theta = p / rho the sound speed
    is cs^2 = theta h'(theta) / (h (h'(theta) - 1)), evaluated here by finite differences of
    the enthalpy alone; cold and hot limits 5/3 theta and 1/3;
  * the inverse theta(h) composed with h(theta) is the identity;
  * con2prim: round trip P -> U -> P, the analytic dp/dxi against a finite difference of
    p(xi), and Newton's quadratic convergence from a close guess (8 iterations suffice);
  * a boosted uniform state stays uniform; a periodic run conserves D, m and tau.
"""
import math

import numpy as np
import pytest

from oracle import Config, Solver
from oracle.physics import SRHD
from paper_2607_19277_gb300 import workloads as W

special = pytest.importorskip("scipy.special")


def _synge_exact(theta):
    return special.kve(3, 1.0 / theta) / special.kve(2, 1.0 / theta)


def test_enthalpy_follows_bessel_definition():
    ph = SRHD(4.0 / 3.0, "synge")
    th = np.logspace(-4, 4, 4001)
    h = ph.enthalpy(np.ones_like(th), th)
    ex = _synge_exact(th)
    assert np.max(np.abs(h / ex - 1.0)) < 0.021
    # both limits exactly: h -> 1 + 5/2 theta (monatomic, gamma 5/3), h -> 4 theta (gamma 4/3)
    for t, f, want in ((1e-6, lambda h, t: (h - 1.0) / t, 2.5), (1e6, lambda h, t: h / t, 4.0)):
        ha = ph.enthalpy(1.0, t)
        he = _synge_exact(np.array([t]))[0]
        assert abs(f(ha, t) - want) < 1e-4 and abs(f(he, t) - want) < 1e-3


def test_theta_of_h_inverts_enthalpy():
    ph = SRHD(4.0 / 3.0, "synge")
    th = np.logspace(-6, 6, 1001)
    back = ph.theta_of_h(ph.enthalpy(1.0, th))
    assert np.max(np.abs(back / th - 1.0)) < 1e-9
    assert ph.theta_of_h(1.0) == 0.0


def test_sound_speed_is_isentropic_derivative():
    ph = SRHD(4.0 / 3.0, "synge")
    th = np.logspace(-4, 4, 801)
    dt = 1e-4 * th       # central difference: truncation ~1e-8, round-off ~1e-12 / 1e-4 h
    hp = (ph.enthalpy(1.0, th + dt) - ph.enthalpy(1.0, th - dt)) / (2.0 * dt)
    h = ph.enthalpy(1.0, th)
    want = th * hp / (h * (hp - 1.0))
    got = ph.sound_speed2(np.ones_like(th), th)
    assert np.max(np.abs(got / want - 1.0)) < 1e-6
    assert np.all(got < 1.0 / 3.0)                                  # causal
    assert abs(ph.sound_speed2(1.0, 1e-7) / 1e-7 - 5.0 / 3.0) < 1e-5  # cold: gamma 5/3
    assert abs(ph.sound_speed2(1.0, 1e7) - 1.0 / 3.0) < 1e-6         # hot: radiation
    # the ideal gas with the same isentropic formula (h' = gamma/(gamma-1)) gives gamma theta/h
    pi = SRHD(1.4)
    assert np.allclose(pi.sound_speed2(1.0, th), 1.4 * th / pi.enthalpy(1.0, th), rtol=1e-14)


def _states(n, seed, theta=(1e-4, 1e3), lor=(1.0, 10.0)):
    rng = np.random.default_rng(seed)
    P = np.zeros((5, n))
    P[0] = rng.uniform(0.01, 10.0, n)
    P[4] = P[0] * np.exp(rng.uniform(math.log(theta[0]), math.log(theta[1]), n))
    g = rng.uniform(lor[0], lor[1], n)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    P[1:4] = np.sqrt(g * g - 1.0) * d
    return P, g


def test_con2prim_round_trip_synge():
    ph = SRHD(4.0 / 3.0, "synge")
    P, g = _states(4000, 3)
    U = ph.prim2cons(P)
    for guess in (None, ph.aux_from_prim(P) * 1.01):
        P2, A = ph.cons2prim(U, guess)
        assert np.max(np.abs(P2[0] - P[0]) / P[0]) < 1e-12
        assert np.max(np.abs(P2[4] - P[4]) / P[4]) < 1e-9
        assert np.max(np.abs(P2[1:4] - P[1:4])) / np.max(np.abs(P[1:4])) < 1e-12
        assert np.max(np.abs(A[1] - g) / g) < 1e-12


def test_pressure_derivative_and_newton_convergence():
    ph = SRHD(4.0 / 3.0, "synge")
    P, _ = _states(500, 4)
    U = ph.prim2cons(P)
    A = ph.aux_from_prim(P)
    D = U[0]
    S2 = (U[1:4] ** 2).sum(axis=0)
    xi = A[0] * 1.05

    def pres(x):
        w = S2 / (x * x)
        return ph._pressure(x, D, w, 1.0 / np.sqrt(1.0 - w))

    p, dp = pres(xi)
    e = 1e-6 * xi
    num = (pres(xi + e)[0] - pres(xi - e)[0]) / (2.0 * e)
    assert np.max(np.abs(dp - num) / (np.abs(num) + 1e-3)) < 1e-6
    # Newton from a guess 0.1% off converges in at most 8 iterations (quadratically)
    ph8 = SRHD(4.0 / 3.0, "synge")
    ph8.max_iter = 8
    P2, _ = ph8.cons2prim(U, A * 1.001)
    assert np.max(np.abs(P2[0] - P[0]) / P[0]) < 1e-12


def test_synge_cold_limit_matches_ideal_five_thirds():
    syn, ide = SRHD(4.0 / 3.0, "synge"), SRHD(5.0 / 3.0)
    P, _ = _states(200, 5, theta=(1e-7, 1e-6), lor=(1.0, 3.0))
    Us, Ui = syn.prim2cons(P), ide.prim2cons(P)
    # h differs by O(theta^2): tau (which carries the thermal energy) to relative O(theta)
    assert np.max(np.abs(Us - Ui) / np.abs(Ui).max(axis=1, keepdims=True)) < 1e-10
    for d in range(3):
        ls, li = syn.lambdas(P, d), ide.lambdas(P, d)
        assert np.max(np.abs(ls[0] - li[0])) < 1e-8 and np.max(np.abs(ls[1] - li[1])) < 1e-8


def test_synge_boosted_uniform_state_is_stationary():
    s = Solver(Config(physics="srhd", eos="synge", limiter="vanleer", flux="tvdlf", rk=3,
                      base_blocks=(1, 1, 1)))
    s.set_state(W.uniform_state([1.3, 2.0, -1.0, 0.5, 0.7]))
    _, _, c0 = s.get_state()
    for _ in range(3):
        s.step()
    _, _, c1 = s.get_state()
    assert np.max(np.abs(c1 - c0) / np.abs(c0).max(axis=(0, 2, 3, 4), keepdims=True)) < 1e-14


def test_synge_conservation_periodic():
    # isotropic cells: on a 2x1x1 mesh of [0,1]^3 (dy = 2 dx) this state drives the
    # floor-free scheme to negative pressure with the ideal gamma = 5/3 gas as well
    s = Solver(Config(physics="srhd", eos="synge", limiter="minmod", flux="tvdlf", rk=2,
                      base_blocks=(2, 2, 2)))
    s.set_state(W.srhd_shells(W.SEED_BASE + 77, 32, lorentz_max=2.0, p_amb=0.1, smooth=True))
    s0 = s.conserved_sums()
    for _ in range(4):
        s.step()
    s1 = s.conserved_sums()
    assert np.max(np.abs(s1 - s0) / np.abs(s0).max()) < 1e-13
