"""GPU parity of SRHD with the approximate Synge-gas EOS (Section 2.3.4): uniform meshes in
FP64 and FP32, a boosted uniform state, an AMR mesh with coarse-fine ghosts and flux fix-up,
and the batched path (each solve equal to the same solve alone)."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import agile, workloads as W
from parity_util import TOL_FP64, gpu_mesh, oracle_solver, rel_l1, run_both

pytestmark = pytest.mark.gpu
PER, OUT, REF = "periodic", "outflow", "reflect"
SYN = dict(physics="srhd", eos="synge", flux="tvdlf")


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, 2e-5)])
def test_synge_shells(rb, tol):
    """Seeded top-hat shells with Lorentz factors up to 5, minmod, SSPRK2; the primitive
    recovery runs in FP64 in both precisions."""
    spec = dict(SYN, limiter="minmod", rk=2, base_blocks=(2, 2, 2))
    ic = W.srhd_shells(W.SEED_BASE + 4, 32, lorentz_max=5.0, p_amb=0.1)
    m, o, g, r, lev, _ = run_both(spec, ic, 3, real_bytes=rb)
    assert rel_l1(g, r).max() < tol
    if rb == 8:
        aux = m.get_aux()
        assert np.max(np.abs(aux - o.get_aux()) / np.abs(o.get_aux())) < 1e-12
    m.close()


def test_synge_vanleer_smooth_outflow_fp64():
    spec = dict(SYN, limiter="vanleer", rk=3, base_blocks=(1, 2, 1), bc=(PER, PER, OUT, OUT, PER, PER))
    m, o, g, r, lev, _ = run_both(spec, W.random_smooth(5, 12, "srhd"), 3)
    assert rel_l1(g, r).max() < TOL_FP64
    m.close()


@pytest.mark.parametrize("rb", [8, 4])
def test_synge_boosted_uniform_state_stationary(rb):
    m = gpu_mesh(dict(SYN, limiter="vanleer", rk=3, base_blocks=(2, 1, 1)), rb)
    m.set_state(W.uniform_state([1.3, 2.0, -1.0, 0.5, 0.7]))
    _, _, c0 = m.get_state()
    for _ in range(3):
        m.step(0.0)
    _, _, c1 = m.get_state()
    scale = np.abs(c0).max(axis=(0, 2, 3, 4), keepdims=True)
    assert np.max(np.abs(c1 - c0) / scale) < (1e-14 if rb == 8 else 1e-6)
    m.close()


def test_synge_amr_steps_match_oracle_and_conserve():
    spec = dict(SYN, limiter="minmod", rk=2, base_blocks=(3, 3, 2), max_level=3,
                bc=(PER,) * 6, refine_vars=(0, 4), refine_weights=(0.5, 0.5))
    base = W.random_smooth(5, 14, "srhd")

    def ic(x, y, z):
        p = base(x, y, z)
        p[1:4] *= 0.3      # mild four-velocities (conserved prolongation of strong states)
        return p
    o = oracle_solver(spec)
    o.set_state(ic)
    m = gpu_mesh(spec)
    m.set_state(ic)
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
    o.set_state_blocks(cons)
    assert sorted(set(o.get_state()[0].tolist())) == [1, 2, 3]
    s0 = m.conserved_sums()
    for _ in range(2):
        dt = o.cfl_dt()
        o.step(dt)
        m.step(dt)
    lev, _, g = m.get_state()
    _, _, r = o.get_state()
    assert rel_l1(g, r, lev, physics="srhd").max() < TOL_FP64
    s1 = m.conserved_sums()
    assert np.max(np.abs(s1 - s0) / np.abs(s0).max()) < 1e-13
    m.close()


@pytest.mark.parametrize("rb", [4, 8])
def test_synge_batch_equals_alone(rb):
    sides = [32, 48, 32]
    bcs = [(PER,) * 6, (OUT,) * 6, (REF,) * 6]
    cfgs = [agile.make_config(physics="srhd", eos="synge", limiter="minmod", flux="tvdlf", rk=2,
                              real_bytes=rb, base_blocks=(s // 16,) * 3, bc=bc)
            for s, bc in zip(sides, bcs)]
    ics = [W.srhd_shells(300 + i, s, lorentz_max=2.0, p_amb=0.1, smooth=True) for i, s in enumerate(sides)]
    b = agile.Batch(cfgs)
    alone = []
    for i in range(len(sides)):
        b.set_state(i, ics[i])
        m = agile.Mesh(cfgs[i])
        m.set_state(ics[i])
        alone.append(m)
    for _ in range(3):
        dts = b.cfl_dt()
        for i, m in enumerate(alone):
            assert dts[i] == m.cfl_dt()
            m.step(0.0)
        b.step()
    b.sync()
    for i, m in enumerate(alone):
        assert np.array_equal(b.get_state(i)[2], m.get_state()[2]), i
        m.close()
    b.close()
