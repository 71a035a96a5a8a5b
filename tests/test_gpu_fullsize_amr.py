"""AMR at the full size of the 5-level Sedov configuration: base 64^3 (4x4x4 blocks of 16^3),
max_level 5 (effective 1024^3), Loehner refinement on density and energy with the initial
condition re-applied during the initial refinement, regrid every 10 steps, HLL, minmod,
SSPRK2. The oracle cannot run this size; the checks are properties that hold at any size:
all five levels are used, mass and energy are conserved to round-off across steps, fix-ups
and regrids (the blast stays inside the box), and the FP32 run agrees with the FP64 run
after both are averaged to the base level."""
import time

import numpy as np
import pytest

from paper_2607_19277_gb300 import agile, workloads as W

pytestmark = pytest.mark.gpu
SPEC = dict(physics="hd", limiter="minmod", flux="hll", rk=2, cfl=0.4, base_blocks=(4, 4, 4),
            xmin=(-0.5,) * 3, xmax=(0.5,) * 3, bc=("outflow",) * 6, max_level=5,
            refine_vars=(0, 4), refine_weights=(0.5, 0.5), refine_tol=0.2)


def _to_base(lev, ijk, cons):
    """Volume average of every leaf onto the 64^3 base grid (16 cells per base block)."""
    out = np.zeros((5, 64, 64, 64))
    for i in range(len(lev)):
        f = 1 << (lev[i] - 1)
        blk = cons[i]
        if f == 1:
            out[:, 16 * ijk[i, 2]:16 * ijk[i, 2] + 16, 16 * ijk[i, 1]:16 * ijk[i, 1] + 16,
                16 * ijk[i, 0]:16 * ijk[i, 0] + 16] += blk
            continue
        n = 16 // f      # base cells covered per block edge (16 fine cells -> n base cells)
        if n == 0:
            continue
        red = blk.reshape(5, n, f, n, f, n, f).mean(axis=(2, 4, 6))
        z0, y0, x0 = (ijk[i, 2] * n, ijk[i, 1] * n, ijk[i, 0] * n)
        out[:, z0:z0 + n, y0:y0 + n, x0:x0 + n] += red
    return out


def _run(rb, steps=30):
    m = agile.Mesh(agile.make_config(real_bytes=rb, **SPEC))
    m.set_state(W.sedov(r0=0.03))
    for _ in range(4):
        m.regrid(init=True)
    s0 = m.conserved_sums()
    t0 = time.perf_counter()
    zones = 0
    for n in range(steps):
        nblk = m.layout()[0]
        m.step(m.cfl_dt())
        zones += nblk * 4096 * 2
        if n % 10 == 9:
            m.regrid()
    m.sync()
    el = time.perf_counter() - t0
    s1 = m.conserved_sums()
    lev, ijk, cons = m.get_state()
    m.close()
    return s0, s1, lev, ijk, cons, zones / el


def test_sedov_five_levels_full_size():
    s0, s1, lev, ijk, cons, zups = _run(8)
    assert set(lev.tolist()) == {1, 2, 3, 4, 5}
    rel = np.abs(s1 - s0) / np.abs(s0).max()
    assert rel[0] < 1e-12 and rel[4] < 1e-12, rel
    # every leaf position is covered exactly once: total volume is the box
    vol = sum(8.0 ** -(l - 1) for l in lev) / 64.0
    assert abs(vol - 1.0) < 1e-12
    s032, s132, lev32, ijk32, cons32, zups32 = _run(4)
    assert abs(s132[0] - s032[0]) / s032[0] < 1e-6
    a = _to_base(lev, ijk, cons)
    b = _to_base(lev32, ijk32, cons32)
    err = np.abs(a - b).sum(axis=(1, 2, 3)) / np.abs(a).sum(axis=(1, 2, 3))
    assert err[0] < 1e-3, err
    print("sedov 5 levels: %d leaves (fp64), %.3g zone-updates/s fp64, %.3g fp32 (incl. regrids)"
          % (len(lev), zups, zups32))
