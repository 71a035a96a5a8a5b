"""GPU parity at the benchmark's full size and launch configuration: 3-D MHD + GLM on a
periodic 256^3 grid of 4096 blocks (Orszag-Tang-like fields, seeded 1% velocity noise,
HLL, van Leer, SSPRK3, CFL 0.4, dt from the device).

The oracle cannot run 16.7 M cells, so sampled blocks are checked one by one: one SSPRK3
step moves information by at most 3 stages x 2 cells = 6 cells < 16, so a block's new
state depends only on its 26 neighbours. The oracle evolves the 3x3x3-block neighbourhood
of each sampled block (periodic on itself, global dt and global c_h from the GPU) and the
centre block must agree. Whole-mesh properties (conservation of rho, m, e, B) are checked
on all 4096 blocks.
"""
import numpy as np
import pytest

from oracle import Config, Solver
from paper_2607_19277_gb300 import agile, workloads as W
from parity_util import TOL_FP32, TOL_FP64, rel_l1

pytestmark = pytest.mark.gpu
N = 256
NB = N // 16
SPEC = dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, cfl=0.4)
SAMPLES = [(0, 0, 0), (15, 15, 15), (7, 3, 11), (15, 0, 8)]


def _wrapped_ic():
    ic = W.orszag_tang_3d(N)

    def f(x, y, z):
        # positions of a neighbourhood that crosses the periodic boundary map back into
        # [0, 1): the seeded perturbation is keyed by the global cell index
        return ic(np.mod(x, 1.0), np.mod(y, 1.0), np.mod(z, 1.0))
    return f


def _oracle_block(centre, dt, ch):
    lo = [(c - 1) / NB for c in centre]
    hi = [(c + 2) / NB for c in centre]
    o = Solver(Config(base_blocks=(3, 3, 3), xmin=tuple(lo), xmax=tuple(hi), **SPEC))
    o.set_state(_wrapped_ic())
    o.step(dt, ch=ch)
    return o.leaves[(1, 1, 1, 1)][:9, 2:18, 2:18, 2:18]


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, TOL_FP32)])
def test_fullsize_mhd_step_sampled_blocks(rb, tol):
    m = agile.Mesh(agile.make_config(real_bytes=rb, base_blocks=(NB,) * 3, **SPEC))
    m.set_state(W.orszag_tang_3d(N))
    s0 = m.conserved_sums()
    smax, cmax = m.max_speeds()
    dt = 0.4 / smax
    assert abs(m.cfl_dt() - dt) <= 1e-15 * dt
    m.step(0.0)                                   # device dt, as the benchmark runs
    lev, ijk, cons = m.get_state()
    s1 = m.conserved_sums()
    m.close()
    # conservation over the whole periodic mesh (psi is damped, not conserved)
    scale = np.abs(s0[:8]).max()
    assert np.max(np.abs(s1[:8] - s0[:8])) <= (1e-13 if rb == 8 else 1e-6) * scale
    index = {tuple(r): i for i, r in enumerate(ijk.tolist())}
    for c in SAMPLES:
        ref = _oracle_block(c, dt, cmax)
        got = cons[index[c]]
        # FP64: psi against its own norm; FP32: psi (zero at t = 0) against c_max sum |B|
        err = rel_l1(got[None], ref[None], physics="mhd", cmax=cmax if rb == 4 else None)
        assert err.max() < tol, (c, err)


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, TOL_FP32)])
def test_fullsize_mhd_five_steps_sampled_blocks(rb, tol):
    """Five SSPRK3 steps at full size, in the launch configuration the benchmark times.
    Five steps move information by at most 5 x 3 x 2 = 30 cells < 32, so a block's state
    depends only on the 5x5x5-block neighbourhood around it; the oracle evolves that
    neighbourhood (periodic on itself, with the GPU's global dt and c_h of every step)."""
    m = agile.Mesh(agile.make_config(real_bytes=rb, base_blocks=(NB,) * 3, **SPEC))
    m.set_state(W.orszag_tang_3d(N))
    hist = []
    for _ in range(5):
        smax, cmax = m.max_speeds()
        dt = m.cfl_dt()
        m.step(dt)
        hist.append((dt, cmax))
    lev, ijk, cons = m.get_state()
    m.close()
    index = {tuple(r): i for i, r in enumerate(ijk.tolist())}
    for c in [(0, 0, 0), (9, 4, 13)]:
        lo = [(ci - 2) / NB for ci in c]
        hi = [(ci + 3) / NB for ci in c]
        o = Solver(Config(base_blocks=(5, 5, 5), xmin=tuple(lo), xmax=tuple(hi), **SPEC))
        o.set_state(_wrapped_ic())
        for dt, ch in hist:
            o.step(dt, ch=ch)
        ref = o.leaves[(1, 2, 2, 2)][:9, 2:18, 2:18, 2:18]
        got = cons[index[c]]
        err = rel_l1(got[None], ref[None], physics="mhd", cmax=hist[-1][1] if rb == 4 else None)
        assert err.max() < tol, (c, err)


def test_largest_uniform_mesh_fp32():
    """512^3 MHD (32768 blocks, about 4.8 GB per FP32 pool): the persistent launch and the
    block tables at eight times the benchmark size; one step conserves rho, m, e and B and
    stays finite, and the conserved sums agree with a host sum of the state."""
    m = agile.Mesh(agile.make_config(real_bytes=4, base_blocks=(32, 32, 32), **SPEC))
    m.set_state(W.orszag_tang_3d(512))
    s0 = m.conserved_sums()
    m.step(0.0)
    s1 = m.conserved_sums()
    scale = np.abs(s0[:8]).max()
    assert np.max(np.abs(s1[:8] - s0[:8])) <= 1e-6 * scale
    _, _, cons = m.get_state()
    m.close()
    assert np.isfinite(cons).all()
    host = cons.sum(axis=(0, 2, 3, 4)) * (1.0 / 512) ** 3
    assert np.max(np.abs(host - s1) / np.abs(s1).max()) < 1e-12
