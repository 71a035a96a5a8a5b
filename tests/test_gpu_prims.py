"""Initial state from host primitives (agile_set_state_prims, agile_batch_set_state_prims)
equals the callback path (agile_set_state) bit for bit for every physics module, on meshes and
on batch solves; wrong block counts are rejected."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import agile, serving, workloads as W

pytestmark = pytest.mark.gpu

CASES = [("hd", dict(flux="hllc"), lambda: W.random_smooth(5, 3, "hd")),
         ("mhd", dict(flux="hll"), lambda: W.orszag_tang_3d(32, seed=5)),
         ("srhd", dict(flux="tvdlf", gamma=4.0 / 3.0),
          lambda: W.srhd_shells(11, 32, lorentz_max=2.0, p_amb=0.1, smooth=True))]


@pytest.mark.parametrize("physics,kw,icf", CASES)
@pytest.mark.parametrize("rb", [8, 4])
def test_prims_equal_callback(physics, kw, icf, rb):
    cfg = agile.make_config(physics=physics, rk=2, real_bytes=rb, base_blocks=(2, 1, 3),
                            xmin=(-0.2, 0.0, 0.1), xmax=(0.8, 0.5, 1.6), **kw)
    ic = icf()
    a = agile.Mesh(cfg)
    a.set_state(ic)
    b = agile.Mesh(cfg)
    b.set_state_prims(agile.prims_of(ic, cfg))
    ga, gb = a.get_state()[2], b.get_state()[2]
    assert np.array_equal(ga, gb)
    a.step(0.0)
    b.step(0.0)
    assert np.array_equal(a.get_state()[2], b.get_state()[2])
    with pytest.raises(agile.AgileError):
        b.set_state_prims(agile.prims_of(ic, cfg)[:-1])
    a.close()
    b.close()


def test_batch_prims_equal_callback():
    cfgs = [serving.scheme(p, 4, s) for p, s in (("mhd", 32), ("mhd", 48))]
    reqs = [serving.Request(rid=i, physics="mhd", side=s, steps=1, seed=900 + i, arrival=0.0)
            for i, s in enumerate((32, 48))]
    a = agile.Batch(cfgs)
    b = agile.Batch(cfgs)
    for i, r in enumerate(reqs):
        a.set_state(i, serving.initial_condition(r))
        b.set_state_prims(i, serving.prepare(r, 4))
    for i in range(2):
        assert np.array_equal(a.get_state(i)[2], b.get_state(i)[2])
    a.close()
    b.close()


@pytest.mark.parametrize("physics,kw,icf", CASES)
def test_page_locked_buffers_transfer_in_place(physics, kw, icf):
    """Page-locked host buffers are read and written in place by the conversion kernels
    (no device staging copy): primitives in, conserved state in and out give the same
    values bit for bit as pageable buffers."""
    import ctypes as C
    import torch
    cfg = agile.make_config(physics=physics, rk=2, real_bytes=4, base_blocks=(2, 1, 3), **kw)
    ic = icf()
    prims = agile.prims_of(ic, cfg)
    pinned = torch.empty(prims.shape, dtype=torch.float64, pin_memory=True).numpy()
    pinned[...] = prims
    a = agile.Mesh(cfg)
    b = agile.Mesh(cfg)
    a.set_state_prims(prims)
    b.set_state_prims(pinned)
    a.step(0.0)
    b.step(0.0)
    ga = a.get_state()[2]
    out = torch.empty(ga.shape, dtype=torch.float64, pin_memory=True).numpy()
    st = b.lib.agile_get_state(b.ptr, None, None, out.ctypes.data_as(C.POINTER(C.c_double)))
    assert st == 0
    assert np.array_equal(out, ga)
    # the state back in from page-locked memory, one more step on both
    a.set_state_blocks(ga)
    b.set_state_blocks(out)
    a.step(0.0)
    b.step(0.0)
    assert np.array_equal(a.get_state()[2], b.get_state()[2])
    a.close()
    b.close()
