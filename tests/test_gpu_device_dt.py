"""The on-device CFL step equals the host-visible one bit for bit.

A step with dt <= 0 takes dt from maxima reduced on the device: fused into the last stage
(HD, MHD), or, for SRHD, in the first stage's primitive-recovery pass of the next step, with
dt set between that pass and the first stage kernel. agile_cfl_dt reduces the same maxima
with the standalone speeds kernel. Two meshes from the same state, one stepped with the
device dt and one with the host's agile_cfl_dt, must therefore stay bit-equal step after
step; the device dt agrees with the oracle's formula through the host value, which the
parity tests pin."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import workloads as W
from parity_util import gpu_mesh

pytestmark = pytest.mark.gpu
OUT, PER, REF = "outflow", "periodic", "reflect"

CASES = [
    ("srhd", 4, dict(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                     base_blocks=(2, 2, 2)), W.srhd_shells(W.SEED_BASE + 81, 32, lorentz_max=3.0, p_amb=0.1)),
    ("srhd", 8, dict(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                     base_blocks=(2, 2, 2), bc=(OUT, OUT, PER, PER, REF, REF)),
     W.srhd_shells(W.SEED_BASE + 82, 32, lorentz_max=3.0, p_amb=0.1)),
    ("mhd", 4, dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 2, 2)),
     W.random_smooth(9, 83, "mhd")),
    ("hd", 8, dict(physics="hd", limiter="vanleer", flux="tvdlf", rk=3, base_blocks=(2, 1, 2)),
     W.random_smooth(5, 84, "hd")),
]


@pytest.mark.parametrize("name,rb,spec,ic", CASES, ids=[c[0] + str(c[1]) for c in CASES])
def test_device_dt_equals_host_cfl_dt(name, rb, spec, ic):
    a = gpu_mesh(spec, real_bytes=rb)
    b = gpu_mesh(spec, real_bytes=rb)
    a.set_state(ic)
    b.set_state(ic)
    for _ in range(4):
        a.step(0.0)                 # device dt
        b.step(b.cfl_dt())          # host dt from the standalone reduction
        assert np.array_equal(a.get_state()[2], b.get_state()[2])
    assert a.cfl_dt() == b.cfl_dt()
    a.close()
    b.close()
