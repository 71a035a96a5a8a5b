"""GPU parity on uniform grids: the CUDA library (C ABI) against the FP64 oracle.

FP64 stencil: relative L1 per variable <= 1e-12 (the bound the FP64 path is held to);
FP32 stencil on smooth runs: <= 1e-5. Every case evolves the same initial condition on
both sides with the same dt per step; sizes span several blocks, ragged block counts,
every boundary kind and all three physics modules.
"""
import numpy as np
import pytest

from paper_2607_19277_gb300 import workloads as W
from parity_util import TOL_FP32, TOL_FP64, gpu_mesh, oracle_solver, psi_self_l1, rel_l1, run_both

pytestmark = pytest.mark.gpu
OUT, PER, REF = "outflow", "periodic", "reflect"


def test_sod_config1_fp64_20_steps():
    """3-D Euler Sod tube, 64^3 as 4x4x4 blocks, PLM minmod, HLL, SSPRK2, CFL 0.4, 20 steps."""
    spec = dict(physics="hd", limiter="minmod", flux="hll", rk=2, cfl=0.4, base_blocks=(4, 4, 4),
                bc=(OUT, OUT, PER, PER, PER, PER))
    m, o, g, r, lev, dts = run_both(spec, W.sod_x, 20)
    err = rel_l1(g, r)
    assert err.max() < TOL_FP64, err
    assert abs(m.cfl_dt() - o.cfl_dt()) <= 1e-13 * o.cfl_dt()
    s_g, s_o = m.conserved_sums(), o.conserved_sums()
    assert np.max(np.abs(s_g - s_o)) <= 1e-13 * np.abs(s_o).max()
    m.close()


@pytest.mark.parametrize("rb", [8, 4])
def test_mhd_orszag_tang_glm(rb):
    """Ideal MHD + GLM, Orszag-Tang-like field with seeded 1% velocity noise, van Leer, HLL,
    SSPRK3, periodic (the 256^3 workload's physics on 32^3).

    FP64: every variable, psi included, within 1e-12 of its own norm. FP32: rho, m, e and B
    within 1e-5; psi starts at zero and after 4 steps holds only the discretisation error of
    div B (sum |psi| is about 2e-4 of c_max sum |B|), so FP32 rounding of the fluxes, relative
    to c_h |B|, is a larger fraction of it: its error is held to 1e-5 of c_max sum |B| and,
    against its own norm, to 2e-4 (measured about 5e-5)."""
    spec = dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 2, 2))
    m, o, g, r, lev, _ = run_both(spec, W.orszag_tang_3d(32), 4, real_bytes=rb)
    if rb == 8:
        err = rel_l1(g, r, physics="mhd")
        assert err.max() < TOL_FP64, err
    else:
        err = rel_l1(g, r, physics="mhd", cmax=o.signal_speeds()[0])
        assert err.max() < TOL_FP32, err
        assert psi_self_l1(g, r) < 2e-4
    m.close()


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, TOL_FP32)])
def test_mhd_psi_of_natural_size_self_normalised(rb, tol):
    """A smooth MHD state whose psi is of order c_h |B| from the start: every variable,
    psi included, within the precision's bound against its own norm (no widened scale)."""
    spec = dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 2, 2))
    m, o, g, r, lev, _ = run_both(spec, W.random_smooth(9, 31, "mhd"), 4, real_bytes=rb)
    err = rel_l1(g, r, physics="mhd")
    assert err.max() < tol, err
    assert psi_self_l1(g, r) < tol
    m.close()


def test_mhd_tvdlf_minmod_fp64():
    spec = dict(physics="mhd", limiter="minmod", flux="tvdlf", rk=2, base_blocks=(2, 1, 2),
                bc=(OUT, OUT, PER, PER, REF, REF))
    m, o, g, r, lev, _ = run_both(spec, W.random_smooth(9, 31, "mhd"), 3)
    assert rel_l1(g, r, physics="mhd").max() < TOL_FP64
    m.close()


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, 2e-5)])
def test_srhd_shell_at_lorentz_factor_near_ten(rb, tol):
    """One periodic shell of the batched workload's family with Lorentz factor 9.5 on 48^3:
    the FP64 Newton recovery at the top of the configured range, both stencils against the
    oracle, and the largest Lorentz factor of the state."""
    spec = dict(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                base_blocks=(3, 3, 3))
    ic = W.srhd_shells(W.SEED_BASE + 71, 48, n_shells=1, lorentz_min=9.5, lorentz_max=9.5, p_amb=1.0,
                       smooth=True, width=2.0, wrap=True, radius=(0.2, 0.35))
    m, o, g, r, lev, _ = run_both(spec, ic, 3, real_bytes=rb)
    assert rel_l1(g, r).max() < tol
    aux = m.get_aux()
    assert aux[:, 1].max() > 8.0          # Lorentz factors near the initial 9.5 remain
    if rb == 8:
        assert np.max(np.abs(aux - o.get_aux()) / np.abs(o.get_aux())) < 1e-12
    m.close()


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, 2e-5)])
def test_srhd_shells(rb, tol):
    """SRHD with seeded shells (Lorentz factors up to 5), LF flux, minmod, SSPRK2; the
    primitive recovery runs in FP64 in both precisions."""
    spec = dict(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                base_blocks=(2, 2, 2))
    ic = W.srhd_shells(W.SEED_BASE + 4, 32, lorentz_max=5.0, p_amb=0.1)
    m, o, g, r, lev, _ = run_both(spec, ic, 3, real_bytes=rb)
    assert rel_l1(g, r).max() < tol
    if rb == 8:
        aux = m.get_aux()
        assert np.max(np.abs(aux - o.get_aux()) / np.abs(o.get_aux())) < 1e-12
    m.close()


def test_srhd_vanleer_smooth_fp64():
    spec = dict(physics="srhd", limiter="vanleer", flux="tvdlf", rk=3, gamma=4.0 / 3.0,
                base_blocks=(1, 2, 1), bc=(PER, PER, OUT, OUT, PER, PER))
    m, o, g, r, lev, _ = run_both(spec, W.random_smooth(5, 12, "srhd"), 3)
    assert rel_l1(g, r).max() < TOL_FP64
    m.close()


@pytest.mark.parametrize("flux,lim,rk", [("hll", "vanleer", 3), ("tvdlf", "minmod", 2),
                                         ("tvdlf", "vanleer", 3)])
def test_hd_ragged_mesh_all_boundaries(flux, lim, rk):
    """6 blocks (3x2x1: a ragged, non-cubic count), reflecting, outflow and periodic faces."""
    spec = dict(physics="hd", limiter=lim, flux=flux, rk=rk, base_blocks=(3, 2, 1),
                bc=(REF, OUT, OUT, REF, PER, PER))
    m, o, g, r, lev, _ = run_both(spec, W.random_smooth(5, 8, "hd"), 4)
    assert rel_l1(g, r).max() < TOL_FP64
    m.close()


def test_single_block_periodic_self_neighbour():
    spec = dict(physics="hd", limiter="vanleer", flux="hll", rk=3, base_blocks=(1, 1, 1))
    m, o, g, r, lev, _ = run_both(spec, W.density_wave((1.0, 1.0, 1.0)), 5)
    assert rel_l1(g, r).max() < TOL_FP64
    m.close()


def test_hd_fp32_smooth_wave():
    spec = dict(physics="hd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 2, 2))
    m, o, g, r, lev, _ = run_both(spec, W.density_wave((1.0, 1.0, 0.0)), 6, real_bytes=4)
    assert rel_l1(g, r).max() < TOL_FP32
    m.close()


def test_device_dt_matches_cfl_dt():
    """agile_step(dt <= 0) takes the CFL step on the device: same result as passing it."""
    spec = dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(1, 1, 2))
    a = gpu_mesh(spec)
    b = gpu_mesh(spec)
    ic = W.orszag_tang_3d(16)
    a.set_state(ic)
    b.set_state(ic)
    for _ in range(3):
        a.step(0.0)
        b.step(b.cfl_dt())
    ga = a.get_state()[2]
    gb = b.get_state()[2]
    assert np.array_equal(ga, gb)
    a.close()
    b.close()


def test_set_get_state_round_trip_and_sums():
    spec = dict(physics="mhd", limiter="vanleer", flux="hll", rk=3, base_blocks=(2, 1, 1))
    o = oracle_solver(spec)
    o.set_state(W.random_smooth(9, 4, "mhd"))
    _, _, cons = o.get_state()
    m = gpu_mesh(spec)
    m.set_state_blocks(cons)
    assert np.array_equal(m.get_state()[2], cons)
    s = m.conserved_sums()
    assert np.max(np.abs(s - o.conserved_sums())) <= 1e-14 * np.abs(s).max()
    m.close()


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, 2e-5)])
def test_hd_hllc_sod_and_smooth(rb, tol):
    """HLLC (hydrodynamics, paper Table 1) against the oracle on Sod and a smooth state."""
    for ic, lim in ((W.sod_x, "minmod"), (W.random_smooth(5, 17, "hd"), "vanleer")):
        spec = dict(physics="hd", limiter=lim, flux="hllc", rk=3, base_blocks=(2, 2, 1),
                    bc=(OUT, OUT, PER, PER, REF, REF))
        m, o, g, r, lev, _ = run_both(spec, ic, 4, real_bytes=rb)
        assert rel_l1(g, r).max() < (tol if ic is not W.sod_x or rb == 8 else 1e-4)
        m.close()


def test_hd_hllc_stationary_contact_exact_on_gpu():
    def ic(x, y, z):
        x = np.asarray(x)
        return np.stack([np.where(x < 0.5, 1.0, 0.2), 0 * x, 0 * x, 0 * x, 1 + 0 * x])
    spec = dict(physics="hd", limiter="minmod", flux="hllc", rk=2, base_blocks=(2, 1, 1),
                bc=(OUT, OUT, PER, PER, PER, PER))
    m = gpu_mesh(spec)
    m.set_state(ic)
    _, _, c0 = m.get_state()
    for _ in range(5):
        m.step(0.0)
    assert np.abs(m.get_state()[2] - c0).max() < 1e-14
    m.close()


@pytest.mark.parametrize("rb,tol", [(8, TOL_FP64), (4, 2e-5)])
def test_srhd_reflecting_walls_through_the_recovery_pass(rb, tol):
    """SRHD reads its halos as primitives from the recovery pass: at reflecting walls on all
    six faces (x/y halos fetched into the ring, z planes loaded directly) the image negates
    the normal component of u = Gamma v as the oracle negates the momentum; a smooth state
    flowing into the walls, against the oracle in both precisions."""
    spec = dict(physics="srhd", limiter="minmod", flux="tvdlf", rk=2, gamma=4.0 / 3.0,
                base_blocks=(2, 2, 2), bc=(REF,) * 6)
    base = W.random_smooth(5, 92, "srhd")

    def ic(x, y, z):
        p = base(x, y, z)
        p[1:4] *= 0.3
        return p
    m, o, g, r, lev, _ = run_both(spec, ic, 4, real_bytes=rb)
    assert rel_l1(g, r).max() < tol
    if rb == 8:
        aux = m.get_aux()
        assert np.max(np.abs(aux - o.get_aux()) / np.abs(o.get_aux())) < 1e-12
    m.close()
