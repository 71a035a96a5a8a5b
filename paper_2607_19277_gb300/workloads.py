"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle's tests.

This module holds no arithmetic of the finite-volume method: it only states initial
conditions as PRIMITIVE fields at cell centres and draws reproducible random numbers.
Each side (the CUDA library, the CPU oracle) converts primitives to conserved variables
with its own code.

Random numbers come from SplitMix64 (Steele, Lea & Flood 2014, "Fast splittable
pseudorandom number generators", OOPSLA), used counter-style: value i of stream `seed`
is mix(seed + (i + 1) * 0x9E3779B97F4A7C15), so any cell can draw its own numbers from
its global index without a sequential state.

Primitive layouts (per cell):
  hd   : rho, vx, vy, vz, p
  mhd  : rho, vx, vy, vz, p, Bx, By, Bz, psi
  srhd : rho, ux, uy, uz, p      (u = Gamma * v, the spatial four-velocity)
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 20260000  # seed = SEED_BASE + workload index


def splitmix64(seed: int, counter) -> np.ndarray:
    """SplitMix64 output for the given counters of stream `seed` (uint64 array)."""
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counter) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, counter) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ----------------------------------------------------------------------------------------
# Initial conditions. Each returns prim[nvar, n] for cell centres x, y, z (1-D arrays).
# ----------------------------------------------------------------------------------------

def sod_x(x, y, z, gamma=5.0 / 3.0, x0=0.5):
    """Sod shock tube along x: (rho, p) = (1, 1) left of x0, (0.125, 0.1) right; v = 0."""
    x = np.asarray(x, dtype=np.float64)
    left = x < x0
    prim = np.zeros((5, x.size))
    prim[0] = np.where(left, 1.0, 0.125)
    prim[4] = np.where(left, 1.0, 0.1)
    return prim


def sod_axis(axis: int, x0=0.5):
    """Sod tube along `axis` (0, 1, 2); the same states as `sod_x`."""
    def ic(x, y, z):
        c = (x, y, z)[axis]
        return sod_x(c, y, z, x0=x0)
    return ic


def density_wave(direction=(1.0, 1.0, 1.0), amp=0.2):
    """Advected density wave rho = 1 + amp sin(2 pi k.x), v = direction, p = 1.

    With periodic boundaries the exact solution at time t is the initial field shifted
    by v t, for any wave vector k = direction (unit-period along each active axis).
    """
    k = np.asarray(direction, dtype=np.float64)

    def ic(x, y, z):
        x = np.asarray(x, dtype=np.float64)
        phase = 2.0 * math.pi * (k[0] * x + k[1] * np.asarray(y) + k[2] * np.asarray(z))
        prim = np.zeros((5, x.size))
        prim[0] = 1.0 + amp * np.sin(phase)
        prim[1] = k[0]
        prim[2] = k[1]
        prim[3] = k[2]
        prim[4] = 1.0
        return prim
    return ic


def density_wave_exact(direction=(1.0, 1.0, 1.0), amp=0.2):
    """Exact density of `density_wave` at time t (cell-centre values)."""
    k = np.asarray(direction, dtype=np.float64)

    def rho(x, y, z, t):
        phase = 2.0 * math.pi * (k[0] * (x - k[0] * t) + k[1] * (y - k[1] * t)
                                 + k[2] * (z - k[2] * t))
        return 1.0 + amp * np.sin(phase)
    return rho


def orszag_tang_3d(n_cells: int, seed: int = SEED_BASE + 2, perturb: float = 0.01):
    """3-D Orszag-Tang-like MHD state on [0,1]^3 (Section 4.5 of the paper, no cooling).

    rho = 4, p = rho T = 1 (T = 0.25), B0 = sqrt(2 p / beta) with beta = 3,
    v = (-sin 2 pi y cos 2 pi z, sin 2 pi x cos 2 pi z, 0),
    B = B0 (-sin 2 pi y cos 2 pi z, sin 4 pi x cos 2 pi z, 0), psi = 0.
    Each velocity component gets perturb * U(-1, 1) * max|v| (max|v| = 1 for this
    pattern), drawn from SplitMix64 keyed by the global cell index at resolution
    n_cells^3 (the uniform grid): counter = 3 * (ix + n (iy + n iz)) + component.
    """
    def ic(x, y, z):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        tp = 2.0 * math.pi
        b0 = math.sqrt(2.0 * 1.0 / 3.0)
        prim = np.zeros((9, x.size))
        prim[0] = 4.0
        prim[1] = -np.sin(tp * y) * np.cos(tp * z)
        prim[2] = np.sin(tp * x) * np.cos(tp * z)
        prim[3] = 0.0
        prim[4] = 1.0
        prim[5] = -b0 * np.sin(tp * y) * np.cos(tp * z)
        prim[6] = b0 * np.sin(2.0 * tp * x) * np.cos(tp * z)
        prim[7] = 0.0
        prim[8] = 0.0
        if perturb:
            ix = np.floor(x * n_cells).astype(np.int64)
            iy = np.floor(y * n_cells).astype(np.int64)
            iz = np.floor(z * n_cells).astype(np.int64)
            cell = (ix + n_cells * (iy + n_cells * iz)).astype(np.uint64)
            for c in range(3):
                r = uniform01(seed, cell * np.uint64(3) + np.uint64(c))
                prim[1 + c] += perturb * (2.0 * r - 1.0) * 1.0
        return prim
    return ic


def sedov(gamma=5.0 / 3.0, energy=1.0, r0=0.03, rho0=1.0, p0=1e-5, centre=(0.0, 0.0, 0.0)):
    """Sedov blast: uniform (rho0, p0), energy deposited as uniform pressure in r < r0.

    The pressure inside is (gamma - 1) energy / (4/3 pi r0^3), so the deposited energy is
    `energy` up to the cell-centre sampling of the sphere; tests take the actual deposit
    from the conserved total.
    """
    p_in = (gamma - 1.0) * energy / (4.0 / 3.0 * math.pi * r0 ** 3)

    def ic(x, y, z):
        x = np.asarray(x, dtype=np.float64)
        r2 = (x - centre[0]) ** 2 + (np.asarray(y) - centre[1]) ** 2 + (np.asarray(z) - centre[2]) ** 2
        prim = np.zeros((5, x.size))
        prim[0] = rho0
        prim[4] = np.where(r2 < r0 * r0, p_in, p0)
        return prim
    return ic


def srhd_shells(seed: int, n_cells: int, n_shells=None, rho_amb=1.0, p_amb=0.01,
                lorentz_max=10.0, smooth=False, width=1.5, lorentz_min=1.0, wrap=False,
                radius=(0.1, 0.3)):
    """SRHD state on [0,1]^3: ambient (rho, p) with 1-3 seeded spherical shells.

    Per shell s (draws 8 s .. 8 s + 7 of the stream): centre U[0,1]^3, radius U[radius],
    rho_shell U[1, 10], radial Lorentz factor U[lorentz_min, lorentz_max]; the shell is
    2 width cells wide (width = 1.5 by default) and moves radially outward with four-velocity
    sqrt(Gamma^2 - 1). smooth=False: a top hat |r - R| < width dx; smooth=True: a Gaussian
    radial profile exp(-(r - R)^2 / (2 (width dx)^2)) of the density excess and of the
    four-velocity (shells combine by the larger weight). wrap=True measures the distance
    to a shell's centre by the periodic minimum image, so that a shell reaching across a
    face of the periodic box continues on the opposite side instead of being cut there.
    """
    if n_shells is None:
        n_shells = 1 + int(uniform01(seed, np.array([1000]))[0] * 3.0)
    shells = []
    for s in range(n_shells):
        u = uniform01(seed, np.arange(8 * s, 8 * s + 8))
        shells.append(dict(c=(u[0], u[1], u[2]), R=radius[0] + (radius[1] - radius[0]) * u[3], rho=1.0 + 9.0 * u[4],
                           lorentz=lorentz_min + (lorentz_max - lorentz_min) * u[5]))
    dx = 1.0 / n_cells

    def ic(x, y, z):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        prim = np.zeros((5, x.size))
        prim[0] = rho_amb
        prim[4] = p_amb
        wmax = np.zeros(x.size)
        for sh in shells:
            ddx, ddy, ddz = x - sh["c"][0], y - sh["c"][1], z - sh["c"][2]
            if wrap:
                ddx, ddy, ddz = (d - np.floor(d + 0.5) for d in (ddx, ddy, ddz))
            r = np.sqrt(ddx * ddx + ddy * ddy + ddz * ddz)
            ur = math.sqrt(sh["lorentz"] ** 2 - 1.0)
            rs = np.where(r > 0, r, 1.0)
            if smooth:
                w = np.exp(-((r - sh["R"]) ** 2) / (2.0 * (width * dx) ** 2))
                take = w > wmax
                wmax = np.where(take, w, wmax)
                prim[0] = np.where(take, rho_amb + (sh["rho"] - rho_amb) * w, prim[0])
                for c, d in enumerate((ddx, ddy, ddz)):
                    prim[1 + c] = np.where(take, w * ur * d / rs, prim[1 + c])
            else:
                inside = np.abs(r - sh["R"]) < width * dx
                prim[0] = np.where(inside, sh["rho"], prim[0])
                for c, d in enumerate((ddx, ddy, ddz)):
                    prim[1 + c] = np.where(inside, ur * d / rs, prim[1 + c])
        return prim
    ic.shells = shells
    return ic


def double_kelvin_helmholtz(rho_in=2.0, rho_out=1.0, v0=0.5, p0=2.5, width=0.02, amp=0.01,
                            seed: int = SEED_BASE + 6):
    """Doubly periodic shear flow on [0,1]^3: v_x = +v0 outside 0.25 < y < 0.75 and -v0
    inside (tanh profiles of the given width), density rho_in inside and rho_out outside,
    uniform pressure, and a small v_y perturbation amp sin(4 pi x) plus a seeded phase per
    z-plane (a stand-in for the double Kelvin-Helmholtz benchmark of Section 3.1, whose
    exact setup is not given)."""
    phase = 2.0 * math.pi * uniform01(seed, np.arange(1))[0]

    def ic(x, y, z):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        inner = 0.5 * (np.tanh((y - 0.25) / width) - np.tanh((y - 0.75) / width))
        prim = np.zeros((5, x.size))
        prim[0] = rho_out + (rho_in - rho_out) * inner
        prim[1] = v0 * (1.0 - 2.0 * inner)
        prim[2] = amp * np.sin(4.0 * math.pi * x + phase) * (1.0 + 0.1 * np.sin(2.0 * math.pi * z))
        prim[4] = p0
        return prim
    return ic


def uniform_state(prim_values):
    """A spatially uniform state with the given primitive vector."""
    pv = np.asarray(prim_values, dtype=np.float64)

    def ic(x, y, z):
        x = np.asarray(x)
        return np.repeat(pv[:, None], x.size, axis=1)
    return ic


def random_smooth(nvar: int, seed: int, kind: str, n_modes: int = 3):
    """Smooth random state (a few seeded Fourier modes) used for parity cases.

    kind 'hd' / 'mhd' / 'srhd' keeps density and pressure positive and, for srhd,
    four-velocities of order one.
    """
    u = uniform01(seed, np.arange(nvar * n_modes * 4))
    amps = u.reshape(nvar, n_modes, 4)

    def ic(x, y, z):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        prim = np.zeros((nvar, x.size))
        for v in range(nvar):
            acc = np.zeros(x.size)
            for m in range(n_modes):
                a, kx, ky, kz = amps[v, m]
                acc += (a - 0.5) * np.sin(2 * math.pi * ((1 + int(3 * kx)) * x
                                                         + (1 + int(3 * ky)) * y
                                                         + (1 + int(3 * kz)) * z) + 7.0 * a)
            prim[v] = acc
        prim[0] = 1.0 + 0.3 * np.tanh(prim[0])
        prim[4] = 1.0 + 0.3 * np.tanh(prim[4])
        if kind == "srhd":
            prim[1:4] *= 1.5
        if kind == "mhd":
            prim[8] = 0.05 * prim[8]
        return prim
    return ic


def skew_normal_cooling(n: int = 256, t_min: float = 1e-2, t_max: float = 1e2, t_peak: float = 0.3,
                        sigma: float = 3.0, skew: float = 7.0, peak: float = 1.0):
    """Tabulated optically thin loss function Lambda(T) in code units (T = p / rho): the
    log-skew-normal shape of the paper's mixing-layer setup,
        Lambda(T) = 2 A / (sigma T) phi((ln T - mu)/sigma) Phi(skew (ln T - mu)/sigma),
    with mu chosen so that the maximum sits at T = t_peak and A so that it equals `peak`.
    Returns (T, Lambda) on n nodes uniformly spaced in ln T over [t_min, t_max].
    The table is an input: both the oracle and the library take it as given."""
    def shape(lnt, mu):
        z = (lnt - mu) / sigma
        phi = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
        big_phi = 0.5 * (1.0 + np.array([math.erf(skew * zi / math.sqrt(2.0)) for zi in np.atleast_1d(z)]))
        return 2.0 / (sigma * np.exp(lnt)) * phi * big_phi.reshape(np.shape(z))

    # argmax of the shape in ln T moves rigidly with mu: locate it once for mu = 0 on a
    # fine grid and shift
    grid = np.linspace(-6.0 * sigma, 6.0 * sigma, 200001)
    g = shape(grid, 0.0)
    mu = math.log(t_peak) - grid[int(np.argmax(g))]
    amp = peak / float(shape(np.array([math.log(t_peak)]), mu)[0])
    lnt = np.linspace(math.log(t_min), math.log(t_max), n)
    lam = amp * shape(lnt, mu)
    if not np.all(lam > 0.0):
        raise ValueError("the loss function underflows to zero on [t_min, t_max]; raise t_min")
    return np.exp(lnt), lam
