"""Batched independent solves: every solve's result is the same alone and in the mix (bit
for bit: the same kernels and per-block arithmetic, each solve with its own CFL dt and GLM
speed), the CUDA-graph replay of later steps equals eager stepping, and one batched solve
matches the FP64 oracle."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import agile, workloads as W
from parity_util import TOL_FP64, oracle_solver, rel_l1

pytestmark = pytest.mark.gpu


def _cfg(side, rb, physics, bc=("periodic",) * 6):
    if physics == "srhd":
        return agile.make_config(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                                 real_bytes=rb, base_blocks=(side // 16,) * 3, bc=bc)
    return agile.make_config(physics="mhd", limiter="vanleer", flux="hll", rk=3, real_bytes=rb,
                             base_blocks=(side // 16,) * 3, bc=bc)


def _ic(physics, seed, side):
    if physics == "srhd":
        # Lorentz factors up to 3: thin (3-cell) shells at Gamma ~ 5 turn unphysical within a
        # step without a floor, in the FP64 oracle as well
        return W.srhd_shells(seed, side, lorentz_max=3.0, p_amb=0.1)
    return W.random_smooth(9, seed, "mhd")


@pytest.mark.parametrize("physics,rb", [("srhd", 4), ("srhd", 8), ("mhd", 4)])
def test_batch_solves_equal_alone(physics, rb):
    sides = [32, 48, 64, 32]
    bcs = [("periodic",) * 6, ("outflow",) * 6, ("periodic",) * 6, ("reflect",) * 6]
    cfgs = [_cfg(s, rb, physics, bc) for s, bc in zip(sides, bcs)]
    b = agile.Batch(cfgs)
    for i, s in enumerate(sides):
        b.set_state(i, _ic(physics, 100 + i, s))
    alone = []
    for i, s in enumerate(sides):
        m = agile.Mesh(cfgs[i])
        m.set_state(_ic(physics, 100 + i, s))
        alone.append(m)
    for step in range(4):
        dts = b.cfl_dt()
        for i, m in enumerate(alone):
            assert dts[i] == m.cfl_dt()
            m.step(0.0)
        b.step()          # step 0 eager, later steps from the captured graph
    b.sync()
    for i, m in enumerate(alone):
        _, _, g = b.get_state(i)
        _, _, a = m.get_state()
        assert np.array_equal(g, a), i
        m.close()
    assert b.launches() > 0
    b.close()


def test_batched_solve_matches_oracle_fp64():
    spec = dict(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                base_blocks=(3, 3, 3))
    cfgs = [_cfg(32, 8, "srhd"), agile.make_config(real_bytes=8, **spec)]
    b = agile.Batch(cfgs)
    ic0 = W.srhd_shells(7, 32, lorentz_max=3.0, p_amb=0.1)
    ic1 = W.srhd_shells(8, 48, lorentz_max=3.0, p_amb=0.1)
    b.set_state(0, ic0)
    b.set_state(1, ic1)
    o = oracle_solver(spec)
    o.set_state(ic1)
    for _ in range(3):
        dt = b.cfl_dt()[1]
        o.step(dt)
        b.step()
    _, _, g = b.get_state(1)
    _, _, r = o.get_state()
    assert rel_l1(g, r).max() < TOL_FP64
    b.close()


@pytest.mark.parametrize("physics", ["srhd", "mhd"])
def test_autotune_keeps_results_and_picks_a_shape(physics):
    """The autotuner times eighteen launch shapes (three staging layouts x three grids x two
    block assignments) without touching the solution; the tuned batch (re-captured graph)
    gives the same results bit for bit as the untuned one."""
    sides = [32, 48, 64]
    cfgs = [_cfg(s, 4, physics) for s in sides]
    a, b = agile.Batch(cfgs), agile.Batch(cfgs)
    for i, s in enumerate(sides):
        a.set_state(i, _ic(physics, 200 + i, s))
        b.set_state(i, _ic(physics, 200 + i, s))
    a.step()
    b.step()
    a.step()                  # graph captured before tuning, replaced after it
    b.step()
    before = [a.get_state(i)[2] for i in range(len(sides))]
    grid, dynamic, ms, layout = a.autotune(trials=2)
    after = [a.get_state(i)[2] for i in range(len(sides))]
    assert all(np.array_equal(x, y) for x, y in zip(after, before))
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert grid in (sms, 2 * sms, 3 * sms) and len(ms) == 18 and all(t > 0 for t in ms)
    assert layout in (1, 2, 3)
    assert min(ms) == ms[6 * (layout - 1) + 2 * (grid // sms - 1) + (0 if dynamic else 1)]
    for _ in range(3):
        a.step()
        b.step()
    for i in range(len(sides)):
        assert np.array_equal(a.get_state(i)[2], b.get_state(i)[2]), i
    a.close()
    b.close()
