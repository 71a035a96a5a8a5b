"""Continuous batching: solves attach to and detach from a running batch without moving the
others. Each solve's result equals the same solve run alone as a mesh, bit for bit, across
detachments, attachments into a hole, attachments that grow the block pool, and a batch that
empties and fills again; a solve of another scheme is refused; a detached index is refused
until it is reused."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import agile, workloads as W

pytestmark = pytest.mark.gpu


def _cfg(side, physics="mhd", rb=4):
    if physics == "srhd":
        return agile.make_config(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                                 real_bytes=rb, base_blocks=(side // 16,) * 3)
    return agile.make_config(physics="mhd", limiter="vanleer", flux="hll", rk=3, real_bytes=rb,
                             base_blocks=(side // 16,) * 3)


def _ic(physics, seed, side):
    if physics == "srhd":
        return W.srhd_shells(seed, side, n_shells=1, lorentz_max=3.0, p_amb=1.0, smooth=True, width=2.0,
                             wrap=True)
    return W.random_smooth(9, seed, "mhd")


class Alone:
    """The same request as its own mesh, stepped with the device dt."""

    def __init__(self, side, physics, rb, seed):
        self.m = agile.Mesh(_cfg(side, physics, rb))
        self.m.set_state(_ic(physics, seed, side))

    def step(self, n):
        for _ in range(n):
            self.m.step(0.0)

    def state(self):
        s = self.m.get_state()[2]
        self.m.close()
        return s


@pytest.mark.parametrize("physics,rb", [("mhd", 4), ("srhd", 4), ("mhd", 8)])
def test_attach_detach_keeps_every_solve_equal_to_alone(physics, rb):
    sides = [32, 48, 32]
    b = agile.Batch([_cfg(s, physics, rb) for s in sides])
    ref = {}
    for i, s in enumerate(sides):
        b.set_state(i, _ic(physics, 300 + i, s))
        ref[i] = Alone(s, physics, rb, 300 + i)
    for _ in range(2):
        b.step()
    for r in ref.values():
        r.step(2)
    # solve 1 (48^3) leaves: its 27 blocks become a hole
    r1 = ref.pop(1)
    _, _, s1 = b.get_state(1)
    assert np.array_equal(s1, r1.state())
    b.detach(1)
    with pytest.raises(agile.AgileError):
        b.get_state(1)
    # a 32^3 solve fills part of the hole (index 1 reused); a 64^3 one does not fit and grows
    # the pool
    j = b.attach(_cfg(32, physics, rb))
    assert j == 1
    b.set_state_prims(j, agile.prims_of(_ic(physics, 310, 32), _cfg(32, physics, rb)))
    ref[j] = Alone(32, physics, rb, 310)
    k = b.attach(_cfg(64, physics, rb))
    assert k == 3
    b.set_state(k, _ic(physics, 311, 64))
    ref[k] = Alone(64, physics, rb, 311)
    for _ in range(3):
        b.step()
    for r in ref.values():
        r.step(3)
    for i, r in ref.items():
        _, _, g = b.get_state(i)
        assert np.array_equal(g, r.state()), i
    b.close()


def test_batch_empties_and_fills_again():
    b = agile.Batch([_cfg(32)])
    b.set_state(0, _ic("mhd", 320, 32))
    b.step()
    b.detach(0)
    b.step()                       # nothing attached: a step does nothing
    i = b.attach(_cfg(48))
    assert i == 0
    b.set_state(i, _ic("mhd", 321, 48))
    a = Alone(48, "mhd", 4, 321)
    for _ in range(2):
        b.step()
    a.step(2)
    assert np.array_equal(b.get_state(i)[2], a.state())
    b.close()


def test_attach_refuses_another_scheme():
    b = agile.Batch([_cfg(32)])
    with pytest.raises(agile.AgileError) as ei:
        b.attach(_cfg(32, "srhd"))
    assert ei.value.status == 1
    with pytest.raises(agile.AgileError):
        b.detach(5)
    b.close()


def test_uniform_solves_come_and_go_beside_a_refined_one():
    """A refined solve (ghost slots, ghost tasks and flux-register fix-ups) stays in the batch
    while uniform solves attach before and after it in the index order and detach again: the
    uniform changes patch only their own table ranges and the work list, the refined solve's
    slot offsets stay valid, and every solve equals its run alone bit for bit."""
    amr = agile.make_config(physics="hd", limiter="minmod", flux="hll", rk=2, real_bytes=8, base_blocks=(2, 2, 2),
                            max_level=3, refine_vars=(0, 4), refine_weights=(0.5, 0.5), refine_tol=0.05)
    uni = agile.make_config(physics="hd", limiter="minmod", flux="hll", rk=2, real_bytes=8, base_blocks=(2, 2, 2))
    ic = {0: W.random_smooth(5, 330, "hd"), 1: W.random_smooth(5, 331, "hd")}
    b = agile.Batch([uni, amr])
    alone = {}
    for i, c in ((0, uni), (1, amr)):
        b.set_state(i, ic[i])
        alone[i] = agile.Mesh(c)
        alone[i].set_state(ic[i])
    flags = np.zeros(b.layout(1)[0], np.int32)
    flags[0] = 1
    assert b.regrid_flags(1, flags) == tuple(alone[1].regrid_flags(flags))

    def both(n):
        for _ in range(n):
            b.step()
            for m in alone.values():
                m.step(0.0)

    both(2)
    # the uniform solve before the refined one leaves, a new one takes its index, another
    # one is appended after the refined one
    _, _, s0 = b.get_state(0)
    assert np.array_equal(s0, alone.pop(0).get_state()[2])
    b.detach(0)
    for i, seed in ((0, 332), (2, 333)):
        j = b.attach(uni)
        assert j == i
        ic[j] = W.random_smooth(5, seed, "hd")
        b.set_state(j, ic[j])
        alone[j] = agile.Mesh(uni)
        alone[j].set_state(ic[j])
    both(3)
    b.detach(2)
    alone.pop(2).close()
    both(2)
    for i, m in alone.items():
        lb, ijkb, cb = b.get_state(i)
        lm, ijkm, cm = m.get_state()
        assert np.array_equal(lb, lm) and np.array_equal(ijkb, ijkm), i
        assert np.array_equal(cb, cm), i
        m.close()
    b.close()


def test_pool_repacks_when_half_empty_and_grows_again():
    """Detaching solves until a pool of more than 4096 blocks is less than 60% used
    repacks it (the live solves copied into a smaller pool), a later attach grows it again; the solves that stay equal
    their runs alone bit for bit throughout."""
    cfg = agile.make_config(physics="hd", limiter="vanleer", flux="tvdlf", rk=3, real_bytes=4,
                            base_blocks=(8, 8, 8))                     # 512 blocks each
    b = agile.Batch([cfg] * 10)
    keep = {1: None, 4: None, 7: None, 9: None}
    for i in range(10):
        b.set_state(i, W.random_smooth(5, 340 + i, "hd"))
    for i in keep:
        keep[i] = agile.Mesh(cfg)
        keep[i].set_state(W.random_smooth(5, 340 + i, "hd"))

    def both(n):
        for _ in range(n):
            b.step()
            for m in keep.values():
                m.step(0.0)

    both(1)
    for i in range(10):            # the fifth detach leaves 2560 of 5120 blocks: repacked
        if i not in keep:          # into 3200 blocks; the sixth leaves a hole
            b.detach(i)
    both(2)
    for seed in (350, 351, 352):   # into the hole, after the last solve, then the pool grows
        j = b.attach(cfg)
        b.set_state(j, W.random_smooth(5, seed, "hd"))
        keep[j] = agile.Mesh(cfg)
        keep[j].set_state(W.random_smooth(5, seed, "hd"))
    both(2)
    for i, m in keep.items():
        assert np.array_equal(b.get_state(i)[2], m.get_state()[2]), i
        m.close()
    b.close()
