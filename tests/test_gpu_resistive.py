"""Resistive MHD (Section 2.3.3: -curl(eta J) in the induction equation, div(B x eta J) in the
energy equation, added as sources of every RK stage with the compact face-neighbour
stencil): parity of the CUDA library with the FP64 oracle on uniform meshes with every
boundary kind, on a three-level mesh (the stencil reads prolonged and restricted face
ghosts), in the FP64 and FP32 stencils, and the diffusive CFL bound. psi is compared
against its own norm (the states start with psi of natural size)."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import workloads as W
from parity_util import TOL_FP32, TOL_FP64, gpu_mesh, oracle_solver, psi_self_l1, rel_l1, run_both

pytestmark = pytest.mark.gpu
OUT, PER, REF = "outflow", "periodic", "reflect"


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, TOL_FP32)])
@pytest.mark.parametrize("limiter,flux", [("vanleer", "hll"), ("minmod", "tvdlf")])
def test_resistive_periodic(rb, tol, limiter, flux):
    spec = dict(physics="mhd", limiter=limiter, flux=flux, rk=3, base_blocks=(2, 2, 2), eta=0.01)
    m, o, g, r, lev, _ = run_both(spec, W.random_smooth(9, 61, "mhd"), 3, real_bytes=rb)
    err = rel_l1(g, r, physics="mhd")
    assert err.max() < tol, err
    assert psi_self_l1(g, r) < tol
    m.close()


def test_resistive_every_boundary_kind_fp64():
    spec = dict(physics="mhd", limiter="vanleer", flux="hll", rk=2, base_blocks=(3, 2, 1), eta=0.02,
                bc=(OUT, OUT, REF, REF, PER, PER))
    m, o, g, r, lev, _ = run_both(spec, W.random_smooth(9, 62, "mhd"), 3)
    assert rel_l1(g, r, physics="mhd").max() < TOL_FP64
    m.close()


def test_resistive_dt_takes_the_diffusive_bound():
    """With a large eta the step is set by 2 eta sum_d dx_d^-2, on both sides."""
    spec = dict(physics="mhd", limiter="vanleer", flux="hll", rk=2, base_blocks=(2, 1, 1), eta=5.0)
    m = gpu_mesh(spec)
    o = oracle_solver(spec)
    ic = W.random_smooth(9, 63, "mhd")
    m.set_state(ic)
    o.set_state(ic)
    smax, _ = m.max_speeds()
    dt = m.cfl_dt()
    assert dt == pytest.approx(o.cfl_dt(), rel=1e-13)
    assert dt < 0.4 / smax
    m.step(0.0)                   # device dt takes the same bound
    o.step(dt)
    _, _, g = m.get_state()
    _, _, r = o.get_state()
    assert rel_l1(g, r, physics="mhd").max() < TOL_FP64
    m.close()


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


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, TOL_FP32)])
def test_resistive_three_level_mesh(rb, tol):
    spec = dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(3, 3, 2), max_level=3,
                bc=(OUT, OUT, PER, PER, REF, REF), eta=0.01)
    ic = W.random_smooth(9, 64, "mhd")
    o = oracle_solver(spec)
    o.set_state(ic)
    m = gpu_mesh(spec, real_bytes=rb)
    m.set_state(ic)
    _force(o, m, {(1, 1, 1, 1)})
    _force(o, m, {(2, 3, 3, 3), (2, 2, 2, 2)})
    _, _, cons = o.get_state()
    m.set_state_blocks(cons)
    for _ in range(2):
        dt = o.cfl_dt()
        assert m.cfl_dt() == pytest.approx(dt, rel=1e-12 if rb == 8 else 1e-5)
        o.step(dt)
        m.step(dt)
    lev, _, g = m.get_state()
    olev, _, r = o.get_state()
    assert np.array_equal(lev, olev) and sorted(set(olev.tolist())) == [1, 2, 3]
    err = rel_l1(g, r, lev, physics="mhd")
    assert err.max() < tol, err
    m.close()
