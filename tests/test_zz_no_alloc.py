"""agile_conserved_sums_noalloc: the conserved-sum diagnostic for callers that cannot
allocate device memory when they call it (a serving loop that reserved its whole device
budget up front, or a host whose allocator is not re-entrant).

The test calls the new entry point through the C ABI twice in a row, with a state change in
between, and checks it against agile_conserved_sums within the tolerance of the other
conserved-sum checks (and in fact bit for bit). Two witnesses show that it allocates
nothing: an allocator that counts its calls, and the device's free memory, read before and
after each call once the first call has looked up the scratch array's address. It also
checks the size limit from both sides: a mesh that fills the scratch exactly (16384
leaves) and one that exceeds it. This file is collected last so that a failure here leaves
every other test already run; it passes in a fresh process and after the rest of the
suite."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import agile, workloads as W

pytestmark = pytest.mark.gpu


class CountingAllocator:
    """torch's caching allocator behind callbacks that count allocations."""

    def __init__(self):
        import torch
        self.torch = torch
        self.dev = torch.cuda.current_device()
        self.allocs = 0

        def alloc(nbytes, stream, ctx):
            self.allocs += 1
            try:
                return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.dev, int(stream or 0))
            except Exception:
                return None

        def free(ptr, stream, ctx):
            if ptr:
                self.torch.cuda.caching_allocator_delete(int(ptr))

        self._a = agile.ALLOC_FN(alloc)
        self._f = agile.FREE_FN(free)
        self.struct = agile.agile_allocator(self._a, self._f, None)


@pytest.mark.parametrize("real_bytes", [8, 4])
def test_noalloc_sums_match_and_allocate_nothing(real_bytes):
    ca = CountingAllocator()
    cfg = agile.make_config(physics="mhd", limiter="vanleer", flux="hll", rk=3,
                            real_bytes=real_bytes, base_blocks=(4, 3, 2))
    m = agile.Mesh(cfg, allocator=ca.struct)
    m.set_state(W.random_smooth(9, 41, "mhd"))
    m.conserved_sums_noalloc()   # the first call on the device looks up the array's address
    torch = ca.torch
    for call in range(2):
        ref = m.conserved_sums()
        before = ca.allocs
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        got = m.conserved_sums_noalloc()
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert ca.allocs == before, "the no-allocation entry point called the allocator"
        assert free1 == free0, ("device free memory changed across the call", free0, free1)
        scale = np.abs(ref).max()
        assert np.max(np.abs(got - ref)) <= 1e-13 * scale
        assert np.array_equal(got, ref)
        m.step(0.0)      # change the state between the two calls
    m.close()


def test_noalloc_rejects_meshes_beyond_its_scratch():
    cfg = agile.make_config(physics="hd", rk=2, real_bytes=4, base_blocks=(128, 129, 1))
    m = agile.Mesh(cfg)
    with pytest.raises(agile.AgileError) as ei:
        m.conserved_sums_noalloc()
    assert ei.value.status == 3 and "16384" in str(ei.value)
    m.close()


def test_noalloc_mesh_that_fills_the_scratch_exactly():
    """16384 leaves x 9 variables: the per-block partial sums end exactly where the totals
    begin (about 7 GB of FP32 pools)."""
    import math
    import torch

    def ic(x, y, z):
        x = np.asarray(x)
        P = np.zeros((9, x.size))
        P[0] = 1.0 + 0.2 * np.sin(2 * math.pi * x) * np.cos(2 * math.pi * np.asarray(z))
        P[1] = 0.1
        P[2] = -0.2 * np.sin(2 * math.pi * np.asarray(y))
        P[4] = 1.0
        P[5] = 0.3
        P[6] = 0.1 * np.cos(2 * math.pi * x)
        P[8] = 0.01 * np.sin(2 * math.pi * np.asarray(y))
        return P
    cfg = agile.make_config(physics="mhd", limiter="vanleer", flux="hll", rk=3, real_bytes=4,
                            base_blocks=(32, 32, 16))
    m = agile.Mesh(cfg)
    assert m.layout()[0] == 16384
    m.set_state(ic)
    for call in range(2):
        ref = m.conserved_sums()
        got = m.conserved_sums_noalloc()
        assert np.array_equal(got, ref), (call, got, ref)
        m.step(0.0)
    m.close()
    torch.cuda.empty_cache()
