"""FP32 HD and MHD stencils, whose x/y faces are solved as packed FP32 pairs (the y-face with
x/y components exchanged) and whose z-faces pair their left and right states: parity with the
FP64 oracle on a three-level mesh with every boundary kind (periodic, outflow, reflecting)
and the coarse-fine flux correction, for both limiters and both fluxes the pairs serve;
conservation on a periodic refined mesh."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import workloads as W
from parity_util import TOL_FP32, gpu_mesh, oracle_solver, rel_l1

pytestmark = pytest.mark.gpu
OUT, PER, REF = "outflow", "periodic", "reflect"


def _force(o, m, refine):
    keys = o.ordered_keys()
    flags = np.array([1 if k in refine else 0 for k in keys], np.int32)
    orig = o.flags

    def forced():
        fl, est = orig()
        for k in fl:
            fl[k] = 1 if k in refine else 0
        return fl, est
    o.flags = forced
    try:
        o.regrid()
    finally:
        o.flags = orig
    m.regrid_flags(flags)


def _three_level(spec, ic):
    o = oracle_solver(spec)
    o.set_state(ic)
    m = gpu_mesh(spec, real_bytes=4)
    m.set_state(ic)
    _force(o, m, {(1, 1, 1, 1)})
    _force(o, m, {(2, 3, 3, 3), (2, 2, 2, 2)})
    lev, ijk, _ = m.get_state()
    olev, oijk, cons = o.get_state()
    assert np.array_equal(lev, olev) and np.array_equal(ijk, oijk)
    assert sorted(set(olev.tolist())) == [1, 2, 3]
    m.set_state_blocks(cons)
    return o, m


@pytest.mark.parametrize("physics", ["hd", "mhd"])
@pytest.mark.parametrize("flux", ["hll", "tvdlf"])
@pytest.mark.parametrize("limiter", ["minmod", "vanleer"])
def test_fp32_pairs_three_levels_all_boundaries(physics, flux, limiter):
    spec = dict(physics=physics, limiter=limiter, flux=flux, rk=3, base_blocks=(3, 3, 2), max_level=3,
                bc=(OUT, OUT, PER, PER, REF, REF))
    nvar = 9 if physics == "mhd" else 5
    o, m = _three_level(spec, W.random_smooth(nvar, 41, physics))
    for _ in range(3):
        dt = o.cfl_dt()
        o.step(dt)
        m.step(dt)
    lev, _, g = m.get_state()
    _, _, r = o.get_state()
    err = rel_l1(g, r, lev, physics=physics, cmax=o.signal_speeds()[0] if physics == "mhd" else None)
    assert err.max() < TOL_FP32, err
    m.close()


@pytest.mark.parametrize("physics", ["hd", "mhd"])
def test_fp32_pairs_conserve_on_periodic_refined_mesh(physics):
    spec = dict(physics=physics, limiter="vanleer", flux="hll", rk=2, base_blocks=(3, 3, 2), max_level=3,
                bc=(PER,) * 6)
    nvar = 9 if physics == "mhd" else 5
    o, m = _three_level(spec, W.random_smooth(nvar, 42, physics))
    s0 = m.conserved_sums()
    for _ in range(4):
        m.step(m.cfl_dt())
    s1 = m.conserved_sums()
    nc = 8 if physics == "mhd" else 5          # psi is damped, not conserved
    scale = np.abs(s0[:nc]).max()
    assert np.max(np.abs(s1[:nc] - s0[:nc])) <= 2e-6 * scale, (s1 - s0)
    m.close()
