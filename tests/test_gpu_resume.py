"""Checkpoint and resume through the C ABI: a run stopped after some steps, its conserved
state read out (agile_get_state) and loaded into a fresh mesh (agile_set_state_blocks),
continues exactly like the uninterrupted run. Bit for bit for hydrodynamics and MHD (the
state determines the CFL step and the GLM speed); for SRHD within the Newton tolerance, since
the auxiliary (xi, Gamma) guesses are not part of the checkpoint and the resumed run starts
each cell's recovery from the bracket midpoint (the converged values agree to about 1e-14)."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import workloads as W
from parity_util import TOL_FP64, gpu_mesh, rel_l1

pytestmark = pytest.mark.gpu


CASES = {
    "hd": (dict(physics="hd", limiter="vanleer", flux="hllc", rk=3, base_blocks=(2, 2, 1),
                bc=("outflow", "outflow", "periodic", "periodic", "reflect", "reflect")),
           W.random_smooth(5, 81, "hd")),
    "mhd": (dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 2, 1)),
            W.random_smooth(9, 82, "mhd")),
    "srhd": (dict(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0, base_blocks=(2, 2, 2)),
             W.srhd_shells(W.SEED_BASE + 83, 32, n_shells=1, lorentz_max=3.0, p_amb=1.0, smooth=True,
                           width=2.0, wrap=True)),
}


@pytest.mark.parametrize("rb", [8, 4])
@pytest.mark.parametrize("physics", ["hd", "mhd", "srhd"])
def test_resume_continues_the_run(physics, rb):
    spec, ic = CASES[physics]
    a = gpu_mesh(spec, real_bytes=rb)
    a.set_state(ic)
    for _ in range(3):
        a.step(0.0)
    _, _, ckpt = a.get_state()
    b = gpu_mesh(spec, real_bytes=rb)
    b.set_state_blocks(ckpt)
    for _ in range(3):
        a.step(0.0)
        b.step(0.0)
    _, _, ga = a.get_state()
    _, _, gb = b.get_state()
    a.close()
    b.close()
    if physics == "srhd":
        assert rel_l1(gb, ga).max() < (TOL_FP64 if rb == 8 else 1e-6)
    else:
        assert np.array_equal(ga, gb)
