"""Helpers shared by the GPU parity tests: one problem description drives both the CUDA
library (through the C ABI) and the FP64 oracle."""
import numpy as np

from oracle import Config, Solver

TOL_FP64 = 1e-12   # relative L1 per variable, FP64 stencil vs FP64 oracle
TOL_FP32 = 1e-5    # relative L1 per variable, FP32 stencil on smooth runs


def oracle_solver(spec):
    return Solver(Config(**spec))


def gpu_mesh(spec, real_bytes=8):
    from paper_2607_19277_gb300 import agile
    return agile.Mesh(agile.make_config(real_bytes=real_bytes, **spec))


def rel_l1(gpu_cons, ora_cons, levels=None, physics="hd", cmax=None):
    """Relative L1 error per variable: sum |a - b| dV / sum |b| dV over the leaves.

    When the reference norm of a variable is below 1e-12 of the density norm (e.g. a
    momentum component that stays zero), the density norm (energy norm for B and psi)
    is the denominator instead. Without cmax every variable, psi included, is normalised
    by its own norm. With cmax given (the FP32 stencil on states whose psi starts at zero)
    psi's denominator is at least c_max * sum |B| dV: psi then holds only the
    discretisation error of div B, a few 1e-4 of c_h |B| in the Orszag-Tang cases, while
    FP32 rounding of the B and psi fluxes is relative to c_h |B|; psi_self_l1 gives the
    self-normalised figure beside it.
    """
    if levels is None:
        w = np.ones(gpu_cons.shape[0])
    else:
        w = 8.0 ** (-(np.asarray(levels) - 1.0))
    wv = w[:, None, None, None, None]
    num = (np.abs(gpu_cons - ora_cons) * wv).sum(axis=(0, 2, 3, 4))
    den = (np.abs(ora_cons) * wv).sum(axis=(0, 2, 3, 4))
    rho = den[0]
    e = den[4]
    out = np.empty_like(num)
    for v in range(len(num)):
        d = den[v]
        if d < 1e-12 * rho:
            d = e if (physics == "mhd" and v >= 5) else rho
        if physics == "mhd" and v == 8 and cmax is not None:
            d = max(d, cmax * (den[5] + den[6] + den[7]))
        out[v] = num[v] / d
    return out


def psi_self_l1(gpu_cons, ora_cons, levels=None):
    """Relative L1 error of the GLM scalar psi against its own norm."""
    w = np.ones(gpu_cons.shape[0]) if levels is None else 8.0 ** (-(np.asarray(levels) - 1.0))
    num = (np.abs(gpu_cons[:, 8] - ora_cons[:, 8]).sum(axis=(1, 2, 3)) * w).sum()
    den = (np.abs(ora_cons[:, 8]).sum(axis=(1, 2, 3)) * w).sum()
    return num / den


def run_both(spec, ic, steps, real_bytes=8, dt_from="gpu"):
    """Evolve the same initial condition on both sides with identical dt per step."""
    m = gpu_mesh(spec, real_bytes)
    m.set_state(ic)
    o = oracle_solver(spec)
    o.set_state(ic)
    dts = []
    for _ in range(steps):
        dt = m.cfl_dt() if dt_from == "gpu" else o.cfl_dt()
        m.step(dt)
        o.step(dt)
        dts.append(dt)
    lev, ijk, g = m.get_state()
    olev, oijk, r = o.get_state()
    assert np.array_equal(lev, olev) and np.array_equal(ijk, oijk)
    return m, o, g, r, lev, dts
