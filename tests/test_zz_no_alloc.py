"""agile_conserved_sums_noalloc: the conserved-sum diagnostic for callers that cannot
allocate device memory when they call it (inside a CUDA stream capture, in a serving loop
that reserved its whole device budget up front, or where the allocator is not re-entrant).

The test calls the new entry point through the C ABI twice in a row, with a state change in
between, and checks it against agile_conserved_sums within the tolerance of the other
conserved-sum checks (and in fact bit for bit), while an allocator that counts its calls
shows that the new entry point allocates nothing. It also checks the size limit. This file
is collected last so that a failure here leaves every other test already run; it passes in
a fresh process and after the rest of the suite."""
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
    for call in range(2):
        ref = m.conserved_sums()
        before = ca.allocs
        got = m.conserved_sums_noalloc()
        assert ca.allocs == before, "the no-allocation entry point called the allocator"
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
