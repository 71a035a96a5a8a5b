"""GPU parity of the radiative losses (Section 2.3.1, Townsend exact integration, Strang
split around each step) with the FP64 oracle: HD and MHD on uniform meshes (FP64 and FP32),
an AMR mesh whose coarse-fine flux fix-up moves the post-step half into its own pass, a
static state against the exact temperature, a table that is not uniform in ln T (binary
search), the temperature floor, and switching the losses off."""
import numpy as np
import pytest

from oracle import Config, Solver
from oracle.cooling import Cooling
from paper_2607_19277_gb300 import agile, workloads as W
from parity_util import TOL_FP32, TOL_FP64, rel_l1

pytestmark = pytest.mark.gpu
PER, OUT, REF = "periodic", "outflow", "reflect"
TAB = W.skew_normal_cooling(n=128, peak=20.0)


def _both(spec, ic, steps, rb=8, table=TAB):
    m = agile.Mesh(agile.make_config(real_bytes=rb, **spec))
    m.set_cooling(*table)
    m.set_state(ic)
    o = Solver(Config(cooling=table, **spec))
    o.set_state(ic)
    for _ in range(steps):
        dt = m.cfl_dt()
        m.step(dt)
        o.step(dt)
    lev, _, g = m.get_state()
    _, _, r = o.get_state()
    return m, o, lev, g, r


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, TOL_FP32)])
def test_hd_wave_with_losses(rb, tol):
    spec = dict(physics="hd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 2, 1))
    m, o, lev, g, r = _both(spec, W.density_wave((1.0, 1.0, 0.0)), 4, rb)
    assert rel_l1(g, r).max() < tol
    # the losses act: total energy falls, mass and momentum stay
    s = m.conserved_sums()
    m.close()
    o2 = Solver(Config(**spec))
    o2.set_state(W.density_wave((1.0, 1.0, 0.0)))
    for _ in range(4):
        o2.step()
    assert s[4] < o2.conserved_sums()[4] * (1 - 1e-4)


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, TOL_FP32)])
def test_mhd_with_losses(rb, tol):
    spec = dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 2, 2))
    m, o, lev, g, r = _both(spec, W.random_smooth(9, 31, "mhd"), 3, rb)
    assert rel_l1(g, r, physics="mhd").max() < tol     # psi against its own norm
    m.close()


def test_amr_with_fixup_and_losses():
    spec = dict(physics="hd", limiter="minmod", flux="hll", rk=2, base_blocks=(3, 3, 2), max_level=3,
                bc=(OUT, OUT, PER, PER, REF, REF), refine_vars=(0, 4), refine_weights=(0.5, 0.5))
    ic = W.random_smooth(5, 3, "hd")
    m = agile.Mesh(agile.make_config(real_bytes=8, **spec))
    m.set_cooling(*TAB)
    m.set_state(ic)
    o = Solver(Config(cooling=TAB, **spec))
    o.set_state(ic)
    for refine in ({(1, 1, 1, 1)}, {(2, 3, 3, 3), (2, 2, 2, 2)}):
        flags = np.array([1 if k in refine else 0 for k in o.ordered_keys()], np.int32)
        orig = o.flags

        def forced(orig=orig, refine=refine):
            fl, est = orig()
            for k in fl:
                fl[k] = 1 if k in refine else 0
            return fl, est
        o.flags = forced
        try:
            ro = o.regrid()
        finally:
            o.flags = orig
        assert tuple(m.regrid_flags(flags)) == tuple(ro)
    _, _, cons = o.get_state()
    m.set_state_blocks(cons)
    for _ in range(2):
        dt = o.cfl_dt()
        assert abs(m.cfl_dt() - dt) <= 1e-13 * dt
        o.step(dt)
        m.step(dt)
    lev, _, g = m.get_state()
    _, _, r = o.get_state()
    assert sorted(set(lev.tolist())) == [1, 2, 3]
    assert rel_l1(g, r, lev).max() < TOL_FP64
    m.close()


@pytest.mark.parametrize("rb,tol", [(8, 1e-13), (4, 2e-6)])
@pytest.mark.parametrize("uniform_table", [True, False])
def test_static_state_exact_temperature(rb, tol, uniform_table):
    T, L = TAB
    if not uniform_table:          # drop every third node: binary-search lookup
        keep = np.ones(T.size, bool)
        keep[1::3] = False
        T, L = T[keep], L[keep]
    cool = Cooling(T, L, 5.0 / 3.0)
    temps = [0.011, 0.05, 0.3, 0.9, 3.0, 40.0, 150.0]   # incl. the floor region and above the table
    for t in temps:
        m = agile.Mesh(agile.make_config(physics="hd", flux="hll", limiter="vanleer", rk=3, real_bytes=rb,
                                         base_blocks=(1, 1, 1)))
        m.set_cooling(T, L)
        m.set_state(W.uniform_state([1.3, 0.0, 0.0, 0.0, 1.3 * t]))
        dt = 0.02
        for _ in range(3):
            m.step(dt)
        _, _, c = m.get_state()
        m.close()
        e = c[0, 4].ravel()
        tn = t
        for _ in range(3):         # two halves per step compose to the full exact step
            tn = cool.cool_temperature(1.3, np.array([tn]), dt)[0]
        want = 1.3 * tn / (2.0 / 3.0)
        assert np.max(np.abs(e - want)) <= tol * want, (t, e[0], want)


def test_floor_and_switch_off():
    # a flat loss function: T falls linearly, by (gamma - 1) rho Lambda per unit time, and
    # stops on the floor T_0 = 0.1 (reached at t = 1.9 / (2/3 * 5) = 0.57)
    spec = dict(physics="hd", flux="hll", limiter="minmod", rk=2, base_blocks=(1, 1, 1))
    m = agile.Mesh(agile.make_config(real_bytes=8, **spec))
    m.set_cooling(np.array([0.1, 10.0]), np.array([5.0, 5.0]))
    m.set_state(W.uniform_state([1.0, 0.0, 0.0, 0.0, 2.0]))
    m.step(0.2)
    _, _, c = m.get_state()
    assert np.allclose(c[0, 4], (2.0 - 2.0 / 3.0 * 5.0 * 0.2) / (2.0 / 3.0), rtol=1e-14)
    for _ in range(4):
        m.step(0.2)
    _, _, c = m.get_state()
    assert np.allclose(c[0, 4], 0.1 / (2.0 / 3.0), rtol=1e-14)
    T, L = TAB
    # switched off: the same run as a mesh without losses, bit for bit
    ic = W.density_wave((1.0, 0.0, 0.0))
    a = agile.Mesh(agile.make_config(real_bytes=8, **spec))
    a.set_cooling(T, L)
    a.set_cooling(None)
    a.set_state(ic)
    b = agile.Mesh(agile.make_config(real_bytes=8, **spec))
    b.set_state(ic)
    for _ in range(3):
        a.step(0.0)
        b.step(0.0)
    assert np.array_equal(a.get_state()[2], b.get_state()[2])
    for mm in (m, a, b):
        mm.close()


def test_invalid_tables_and_physics_rejected():
    m = agile.Mesh(agile.make_config(physics="hd", base_blocks=(1, 1, 1)))
    T, L = TAB
    for bad_t, bad_l in ((T[::-1], L), (T, -L), (T[:1], L[:1])):
        with pytest.raises(RuntimeError):
            m.set_cooling(bad_t, bad_l)
    m.close()
    s = agile.Mesh(agile.make_config(physics="srhd", flux="tvdlf", gamma=4.0 / 3.0, base_blocks=(1, 1, 1)))
    with pytest.raises(RuntimeError):
        s.set_cooling(T, L)
    s.close()
