"""Closed-form and quasi-closed-form solutions used to pin the oracle.

TEST INFRASTRUCTURE ONLY.

* Exact Riemann solver for the 1-D Euler equations of an ideal gas (Toro 2009,
  "Riemann Solvers and Numerical Methods for Fluid Dynamics", 3rd ed., chapter 4):
  the star pressure is the root of f_L(p) + f_R(p) + (u_R - u_L) = 0 with the shock
  branch f_K = (p - p_K) sqrt(A_K / (p + B_K)), A_K = 2/((gamma+1) rho_K),
  B_K = (gamma-1)/(gamma+1) p_K, and the rarefaction branch
  f_K = 2 c_K/(gamma-1) ((p/p_K)^((gamma-1)/(2 gamma)) - 1); the solution is then sampled
  along x/t.
* Sedov-Taylor point blast (Sedov 1959): R(t) = xi0 (E t^2 / rho0)^(1/5); xi0 follows
  from the energy integral of the self-similar solution, obtained here by integrating the
  similarity ODEs from the strong-shock jump conditions inward.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:
        a = 2.0 / ((g + 1.0) * rho)
        b = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(a / (p + b))
        df = math.sqrt(a / (b + p)) * (1.0 - 0.5 * (p - pk) / (b + p))
    else:
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def riemann_star(rl, ul, pl, rr, ur, pr, g):
    """Star-region pressure and velocity (Newton on the pressure function)."""
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, cl, g)
        fr, dfr = _fk(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_sample(rl, ul, pl, rr, ur, pr, g, s):
    """Exact (rho, u, p) at the similarity coordinates s = (x - x0) / t (numpy array)."""
    ps, us = riemann_star(rl, ul, pl, rr, ur, pr, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    gm = (g - 1.0) / (g + 1.0)
    s = np.asarray(s, dtype=np.float64)
    rho = np.empty_like(s)
    u = np.empty_like(s)
    p = np.empty_like(s)
    for i, si in enumerate(s.ravel()):
        if si <= us:   # left of contact
            if ps > pl:   # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if si <= sl:
                    r, v, q = rl, ul, pl
                else:
                    r = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                    v, q = us, ps
            else:         # left rarefaction
                shl = ul - cl
                cml = cl * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - cml
                if si <= shl:
                    r, v, q = rl, ul, pl
                elif si >= stl:
                    r = rl * (ps / pl) ** (1.0 / g)
                    v, q = us, ps
                else:
                    v = 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + si)
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - si))
                    r = rl * (c / cl) ** (2.0 / (g - 1))
                    q = pl * (c / cl) ** (2.0 * g / (g - 1))
        else:          # right of contact
            if ps > pr:   # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if si >= sr:
                    r, v, q = rr, ur, pr
                else:
                    r = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                    v, q = us, ps
            else:         # right rarefaction
                shr = ur + cr
                cmr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + cmr
                if si >= shr:
                    r, v, q = rr, ur, pr
                elif si <= str_:
                    r = rr * (ps / pr) ** (1.0 / g)
                    v, q = us, ps
                else:
                    v = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + si)
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - si))
                    r = rr * (c / cr) ** (2.0 / (g - 1))
                    q = pr * (c / cr) ** (2.0 * g / (g - 1))
        rho.flat[i], u.flat[i], p.flat[i] = r, v, q
    return rho, u, p


def sedov_xi0(g: float) -> float:
    """Sedov-Taylor constant xi0 for a spherical blast in a uniform gas.

    Self-similar form r = eta R(t), R ~ t^(2/5), v = R' f(eta), rho = rho0 g(eta),
    p = rho0 R'^2 h(eta). Mass, momentum and entropy conservation give, with w = f - eta,
      w g' + g f' = -2 g f / eta,   w f' + h'/g = 3 f / 2,   w (h'/h - gamma g'/g) = 3,
    integrated inward from the strong-shock values f = 2/(gamma+1),
    g = (gamma+1)/(gamma-1), h = 2/(gamma+1) at eta = 1. With R' = 2R/(5t) the energy
    E = 4 pi rho0 R'^2 R^3 I, I = int_0^1 (g f^2 / 2 + h/(gamma-1)) eta^2 d eta,
    so xi0 = (25 / (16 pi I))^(1/5).
    """
    from scipy.integrate import solve_ivp

    def rhs(eta, y):
        f, gg, h = y
        w = f - eta
        a = (1.5 * f - (h / (gg * w)) * (3.0 - 2.0 * g * f / eta)) / (w - g * h / (gg * w))
        dg = -gg * (2.0 * f / eta + a) / w
        dh = h * (3.0 / w + g * dg / gg)
        return [a, dg, dh]

    y0 = [2.0 / (g + 1.0), (g + 1.0) / (g - 1.0), 2.0 / (g + 1.0)]
    sol = solve_ivp(rhs, (1.0, 1e-6), y0, method="DOP853", rtol=1e-11, atol=1e-14,
                    dense_output=True)
    eta = np.linspace(1e-6, 1.0, 200001)
    f, gg, h = sol.sol(eta)
    integrand = (0.5 * gg * f * f + h / (g - 1.0)) * eta * eta
    integral = float(np.trapezoid(integrand, eta))
    return (25.0 / (16.0 * math.pi * integral)) ** 0.2
