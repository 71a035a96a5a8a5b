"""Device-side error reporting: unphysical states and a primitive recovery that cannot
converge latch a status word that the next synchronising call returns; the context stays
usable afterwards. No fault, trap or hang is involved: the kernels only compute NaNs or
flag bad values."""
import numpy as np
import pytest

from paper_2607_19277_gb300 import agile
from parity_util import gpu_mesh

pytestmark = pytest.mark.gpu


def test_negative_pressure_reported():
    spec = dict(physics="hd", base_blocks=(1, 1, 1))
    m = gpu_mesh(spec)
    cons = np.zeros((1, 5, 16, 16, 16))
    cons[:, 0] = 1.0
    cons[:, 4] = -1.0          # e < 0 -> p < 0
    m.set_state_blocks(cons)
    with pytest.raises(agile.AgileError) as ei:
        m.cfl_dt()
    assert ei.value.status == 6     # AGILE_EUNPHYS
    # the mesh and the context still work
    cons[:, 4] = 2.0
    m.set_state_blocks(cons)
    assert m.cfl_dt() > 0
    m.close()


def test_srhd_recovery_failure_reported():
    spec = dict(physics="srhd", flux="tvdlf", gamma=4.0 / 3.0, base_blocks=(1, 1, 1))
    m = gpu_mesh(spec)
    cons = np.zeros((1, 5, 16, 16, 16))
    cons[:, 0] = 1.0
    cons[:, 4] = -3.0          # tau + D < 0: no root in the bracket
    m.set_state_blocks(cons)
    with pytest.raises(agile.AgileError) as ei:
        m.cfl_dt()
    assert ei.value.status in (5, 6)
    m.close()


def test_regrid_flags_length_checked_and_mesh_reusable():
    spec = dict(physics="hd", base_blocks=(2, 1, 1), max_level=2,
                bc=("outflow",) * 2 + ("periodic",) * 4)
    m = gpu_mesh(spec)
    cons = np.ones((2, 5, 16, 16, 16))
    cons[:, 1:4] = 0.0
    m.set_state_blocks(cons)
    with pytest.raises(agile.AgileError):
        m.set_state_blocks(cons[:1])
    assert m.regrid_flags([1, 0]) == (1, 0)
    assert m.layout()[0] == 9
    m.close()


def test_bounded_wait_times_out_and_context_survives():
    """A device wait on a barrier that nothing completes gives up after its poll limit and
    reports AGILE_ETIMEOUT; the same process keeps working afterwards."""
    import ctypes as C
    lib = agile.load()
    flag = C.c_int(-1)
    st = lib.agile_selftest_bounded_wait(None, 4096, C.byref(flag))
    assert st == 7 and flag.value == 1
    spec = dict(physics="hd", base_blocks=(1, 1, 1))
    m = gpu_mesh(spec)
    cons = np.ones((1, 5, 16, 16, 16))
    cons[:, 1:4] = 0.0
    m.set_state_blocks(cons)
    m.step(m.cfl_dt())
    m.sync()
    m.close()
