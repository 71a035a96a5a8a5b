"""Batched solves on refined meshes: one persistent launch per RK stage over the blocks of
all levels of all solves, with the coarse-fine ghost fill and flux fix-up of every solve in
shared launches. Each solve, regridded inside the batch (forced flags or the Loehner
estimate), must equal the same solve run alone as a mesh with the same regrids, bit for
bit, and conserve what it conserves alone."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import agile, workloads as W

pytestmark = pytest.mark.gpu
OUT, PER, REF = "outflow", "periodic", "reflect"


def _cfgs(physics, rb):
    flux = "hll" if physics in ("hd", "mhd") else "tvdlf"
    base = dict(physics=physics, limiter="minmod", flux=flux, rk=2 if physics != "mhd" else 3, real_bytes=rb,
                max_level=3, refine_vars=(0, 4), refine_weights=(0.5, 0.5), refine_tol=0.05)
    if physics == "srhd":
        base["gamma"] = 4.0 / 3.0
    return [agile.make_config(base_blocks=(2, 2, 2), bc=(PER,) * 6, **base),
            agile.make_config(base_blocks=(3, 2, 2), bc=(OUT, OUT, PER, PER, REF, REF), **base),
            agile.make_config(base_blocks=(2, 3, 1), bc=(REF,) * 6, **base)]


def _ic(physics, i):
    nvar = {"hd": 5, "mhd": 9, "srhd": 5}[physics]
    base = W.random_smooth(nvar, 40 + i, physics)
    if physics != "srhd":
        return base

    def f(x, y, z):
        p = base(x, y, z)
        p[1:4] *= 0.3
        return p
    return f


@pytest.mark.parametrize("physics,rb", [("hd", 8), ("hd", 4), ("mhd", 4), ("srhd", 8)])
def test_amr_batch_equals_alone(physics, rb):
    cfgs = _cfgs(physics, rb)
    b = agile.Batch(cfgs)
    alone = []
    for i, c in enumerate(cfgs):
        b.set_state(i, _ic(physics, i))
        m = agile.Mesh(c)
        m.set_state(_ic(physics, i))
        alone.append(m)

    def both_step(n):
        for _ in range(n):
            b.step()
            for m in alone:
                m.step(0.0)

    both_step(2)
    # solve 0: forced refinement of its first block, then of one of the new children
    n0 = b.layout(0)[0]
    flags = np.zeros(n0, np.int32)
    flags[0] = 1
    assert b.regrid_flags(0, flags) == tuple(alone[0].regrid_flags(flags))
    n0 = b.layout(0)[0]
    flags = np.zeros(n0, np.int32)
    flags[-1] = 1
    assert b.regrid_flags(0, flags) == tuple(alone[0].regrid_flags(flags))
    both_step(3)
    # solves 1 and 2: the estimate decides (init re-applies the initial condition)
    assert b.regrid(1, init=True) == tuple(alone[1].regrid(init=True))
    assert b.regrid(2) == tuple(alone[2].regrid())
    both_step(3)
    # every solve at once, one new layout of the pools
    counts = [tuple(m.regrid()) for m in alone]
    assert b.regrid(-1) == (sum(c[0] for c in counts), sum(c[1] for c in counts))
    both_step(2)
    levels = set()
    for i, m in enumerate(alone):
        lb, ijkb, cb = b.get_state(i)
        lm, ijkm, cm = m.get_state()
        assert np.array_equal(lb, lm) and np.array_equal(ijkb, ijkm), i
        assert np.array_equal(cb, cm), i
        levels |= set(lb.tolist())
        m.close()
    assert max(levels) == 3                           # refined twice somewhere
    b.close()


def test_amr_batch_conserves_and_coarsens():
    cfgs = _cfgs("hd", 8)[:1]
    b = agile.Batch(cfgs)
    b.set_state(0, W.random_smooth(5, 41, "hd"))
    n = b.layout(0)[0]
    b.regrid_flags(0, np.ones(n, np.int32))            # every block refined
    assert b.layout(0)[0] == 8 * n
    lev, _, c0 = b.get_state(0)
    w = 8.0 ** -(lev - 1.0)
    m0 = (c0[:, 0].sum(axis=(1, 2, 3)) * w).sum()
    for _ in range(4):
        b.step()
    lev, _, c1 = b.get_state(0)
    m1 = (c1[:, 0].sum(axis=(1, 2, 3)) * w).sum()
    assert abs(m1 - m0) < 1e-13 * m0
    b.regrid_flags(0, -np.ones(8 * n, np.int32))      # and coarsened back
    assert b.layout(0)[0] == n
    b.step()
    b.close()


@pytest.mark.parametrize("physics,rb", [("hd", 4), ("srhd", 8)])
def test_autotune_on_refined_solves(physics, rb):
    """The autotuner's trial launches of the first stage on a batch with coarse-fine faces
    fill the ghost slots from U^n and read them as the first stage does, without touching
    the solution: the tuned batch then steps bit for bit like an untuned one."""
    cfgs = _cfgs(physics, rb)
    a = agile.Batch(cfgs)
    b = agile.Batch(cfgs)
    for i in range(len(cfgs)):
        a.set_state(i, _ic(physics, i))
        b.set_state(i, _ic(physics, i))
    for bb in (a, b):
        n0 = bb.layout(0)[0]
        flags = np.zeros(n0, np.int32)
        flags[0] = 1
        bb.regrid_flags(0, flags)
        bb.step()
    before = [a.get_state(i)[2] for i in range(len(cfgs))]
    a.autotune(trials=2)
    assert all(np.array_equal(a.get_state(i)[2], x) for i, x in enumerate(before))
    for _ in range(2):
        a.step()
        b.step()
    for i in range(len(cfgs)):
        assert np.array_equal(a.get_state(i)[2], b.get_state(i)[2]), i
    a.close()
    b.close()
