"""Oracle physics modules: conserved <-> primitive maps, physical fluxes, signal speeds.

TEST INFRASTRUCTURE ONLY. This package is the plain FP64 CPU oracle that the CUDA path is
checked against; only tests, the smoke check and the bench's CPU-baseline leg use it.
It shares no code with the CUDA library.

Every function works on numpy arrays shaped (nvar, ...) with the variable axis first and
follows the paper's Section 2.3:
  * hd   : Eqs. 2-4 and the closure e = p/(gamma-1) + rho v^2/2 (Section 2.3.1); the
           flux is the HD get_flux of the paper's flux listing (Section 2.3).
  * mhd  : Eqs. 11-13 with GLM (Eq. 14), e = p/(gamma-1) + rho v^2/2 + B^2/2 (units absorb
           4 pi), Section 2.3.3.
  * srhd : Eqs. 15-20, con2prim as a 1-D root find in xi = Gamma^2 rho h (Section
           2.3.4), closed by the ideal-gas enthalpy (Eq. 21) or by the Synge gas (Eq. 22)
           in Mathews' approximation, which Section 2.3.4 names instead of the Bessel
           functions: h = 5/2 theta + sqrt(9/4 theta^2 + 1), theta = p / rho.
  * ffhd : Section 2.3.2, Eqs. 7-9 (frozen-field hydrodynamics along a frozen unit field).
"""
from __future__ import annotations

import numpy as np


class HD:
    """Newtonian hydrodynamics, U = (rho, m, e), P = (rho, v, p)."""

    name = "hd"
    nvar = 5
    naux = 0
    glm = False

    def __init__(self, gamma: float):
        self.gamma = float(gamma)

    def prim2cons(self, P):
        g = self.gamma
        rho, v, p = P[0], P[1:4], P[4]
        U = np.empty_like(P)
        U[0] = rho
        U[1:4] = rho * v
        U[4] = p / (g - 1.0) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])
        return U

    def cons2prim(self, U, aux=None):
        g = self.gamma
        P = np.empty_like(U)
        rho = U[0]
        v = U[1:4] / rho
        P[0] = rho
        P[1:4] = v
        P[4] = (g - 1.0) * (U[4] - 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]))
        return P, None

    def flux(self, P, U, d):
        """Physical flux along axis d from primitives (paper's HD get_flux listing)."""
        g = self.gamma
        rho, v, p = P[0], P[1:4], P[4]
        vd = v[d]
        F = np.empty_like(P)
        F[0] = rho * vd
        for i in range(3):
            F[1 + i] = rho * v[i] * vd
        F[1 + d] = F[1 + d] + p
        F[4] = vd * (p / (g - 1.0) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) + p)
        return F

    def sound_speed(self, P):
        return np.sqrt(self.gamma * P[4] / P[0])

    def lambdas(self, P, d):
        """Smallest and largest characteristic speed along d: v_d -/+ c_s."""
        c = self.sound_speed(P)
        return P[1 + d] - c, P[1 + d] + c


class MHD:
    """Ideal MHD with GLM divergence cleaning, U = (rho, m, e, B, psi)."""

    name = "mhd"
    nvar = 9
    naux = 0
    glm = True

    def __init__(self, gamma: float):
        self.gamma = float(gamma)

    def prim2cons(self, P):
        g = self.gamma
        rho, v, p, B = P[0], P[1:4], P[4], P[5:8]
        U = np.empty_like(P)
        U[0] = rho
        U[1:4] = rho * v
        v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2]
        b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2]
        U[4] = p / (g - 1.0) + 0.5 * rho * v2 + 0.5 * b2
        U[5:8] = B
        U[8] = P[8]
        return U

    def cons2prim(self, U, aux=None):
        g = self.gamma
        P = np.empty_like(U)
        rho = U[0]
        v = U[1:4] / rho
        B = U[5:8]
        v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2]
        b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2]
        P[0] = rho
        P[1:4] = v
        P[4] = (g - 1.0) * (U[4] - 0.5 * rho * v2 - 0.5 * b2)
        P[5:8] = B
        P[8] = U[8]
        return P, None

    def flux(self, P, U, d, ch):
        """Flux along d of Eqs. 11-13; GLM pair F(B_d) = psi, F(psi) = c_h^2 B_d (Eq. 14)."""
        rho, v, p, B, psi = P[0], P[1:4], P[4], P[5:8], P[8]
        vd, Bd = v[d], B[d]
        b2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2]
        ptot = p + 0.5 * b2
        vB = v[0] * B[0] + v[1] * B[1] + v[2] * B[2]
        F = np.empty_like(P)
        F[0] = rho * vd
        for i in range(3):
            F[1 + i] = rho * v[i] * vd - B[i] * Bd
        F[1 + d] = F[1 + d] + ptot
        F[4] = vd * (U[4] + ptot) - Bd * vB
        for i in range(3):
            F[5 + i] = vd * B[i] - Bd * v[i]
        F[5 + d] = psi
        F[8] = ch * ch * Bd
        return F

    def fast_speed(self, P, d):
        """Fast magnetosonic speed along d."""
        rho, p, B = P[0], P[4], P[5:8]
        a2 = self.gamma * p / rho
        b2 = (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / rho
        bd2 = B[d] * B[d] / rho
        s = a2 + b2
        return np.sqrt(0.5 * (s + np.sqrt(s * s - 4.0 * a2 * bd2)))

    def lambdas(self, P, d):
        cf = self.fast_speed(P, d)
        return P[1 + d] - cf, P[1 + d] + cf

    def resistive_source(self, B, dx, eta):
        """Resistive terms of Section 2.3.3 as cell-centred sources on a block interior.

        The induction equation carries -curl(eta J) and the energy equation
        div(B x eta J), J = curl B, with uniform eta. With div B = 0 these are eta lap B and
        eta (J.J + B . lap B): the Ohmic heating eta J^2 plus the change of the magnetic
        energy B . dB/dt. Both are evaluated with the compact second-order stencil over the
        six face neighbours: lap_d a = ((a_+ - a_0) - (a_0 - a_-)) / dx_d^2 and
        d_d a = (a_+ - a_-) / (2 dx_d) (the grad(div B) part of -curl curl B, which needs
        edge neighbours, is the divergence error GLM controls and is not taken).
        B: (3, 20, 20, 20) primitives [z, y, x] with filled face ghosts.
        Returns (S_B (3, 16, 16, 16), S_e (16, 16, 16))."""
        I = slice(2, 18)

        def sl(d, o):
            r = [I, I, I]
            r[2 - d] = slice(2 + o, 18 + o)
            return tuple(r)

        def d1(a, d):
            return (a[sl(d, 1)] - a[sl(d, -1)]) / (2.0 * dx[d])

        def d2(a, d):
            return ((a[sl(d, 1)] - a[sl(d, 0)]) - (a[sl(d, 0)] - a[sl(d, -1)])) / (dx[d] * dx[d])

        lap = np.stack([(d2(B[i], 0) + d2(B[i], 1)) + d2(B[i], 2) for i in range(3)])
        J = np.stack([d1(B[2], 1) - d1(B[1], 2),
                      d1(B[0], 2) - d1(B[2], 0),
                      d1(B[1], 0) - d1(B[0], 1)])
        Bc = B[(slice(None), I, I, I)]
        jj = (J[0] * J[0] + J[1] * J[1]) + J[2] * J[2]
        blap = (Bc[0] * lap[0] + Bc[1] * lap[1]) + Bc[2] * lap[2]
        return eta * lap, eta * (jj + blap)

    def glm_interface(self, PL, PR, d, ch):
        """Exact solution of the linear (B_d, psi) subsystem at a face (Dedner et al. 2002).

        The GLM system of Eq. 14 with flux c_h^2 B_d for psi and psi for B_d has speeds
        +/- c_h; its Riemann solution gives one interface value of B_d and psi, which both
        face states then carry, so the face flux of B_d is psi* and of psi is c_h^2 B_d*.
        """
        bl, br = PL[5 + d], PR[5 + d]
        pl, pr = PL[8], PR[8]
        bstar = 0.5 * (bl + br) - 0.5 * (pr - pl) / ch
        pstar = 0.5 * (pl + pr) - 0.5 * ch * (br - bl)
        PL = PL.copy()
        PR = PR.copy()
        PL[5 + d] = bstar
        PR[5 + d] = bstar
        PL[8] = pstar
        PR[8] = pstar
        return PL, PR


class SRHD:
    """Special-relativistic hydro, U = (D, m, tau), P = (rho, u = Gamma v, p), A = (xi, Gamma).

    eos = "ideal": h = 1 + gamma/(gamma-1) theta (Eq. 21).
    eos = "synge": Mathews' approximation of the Synge gas (Eq. 22 without the Bessel
    functions): h = 5/2 theta + sqrt(9/4 theta^2 + 1). It tends to the ideal gas with
    gamma = 5/3 as theta -> 0 and to gamma = 4/3 as theta -> infinity; gamma is unused.
    """

    name = "srhd"
    nvar = 5
    naux = 2
    glm = False
    max_iter = 50
    tol = 1e-14

    def __init__(self, gamma: float, eos: str = "ideal"):
        if eos not in ("ideal", "synge"):
            raise ValueError("eos must be 'ideal' or 'synge'")
        self.gamma = float(gamma)
        self.eos = eos

    def enthalpy(self, rho, p):
        """Specific enthalpy h(rho, p): Eq. 21 (ideal gas) or the approximate Synge gas."""
        theta = p / rho
        if self.eos == "synge":
            return 2.5 * theta + np.sqrt(2.25 * theta * theta + 1.0)
        g = self.gamma
        return 1.0 + g / (g - 1.0) * theta

    def theta_of_h(self, h):
        """Inverse of h(theta) for the approximate Synge gas: (h - 5/2 theta)^2 =
        9/4 theta^2 + 1 gives 4 theta^2 - 5 h theta + h^2 - 1 = 0; the root with theta = 0
        at h = 1 is theta = (5 h - sqrt(9 h^2 + 16)) / 8."""
        return (5.0 * h - np.sqrt(9.0 * h * h + 16.0)) / 8.0

    def sound_speed2(self, rho, p):
        """Squared sound speed: gamma p / (rho h) (ideal gas); for the approximate Synge
        gas theta (5 h - 8 theta) / (3 h (h - theta)) (the isentropic derivative dp/de
        of that enthalpy, as in Mignone & McKinney 2007)."""
        h = self.enthalpy(rho, p)
        theta = p / rho
        if self.eos == "synge":
            return theta * (5.0 * h - 8.0 * theta) / (3.0 * h * (h - theta))
        return self.gamma * theta / h

    def prim2cons(self, P):
        """Eq. 18 evaluated from the primitives of Eq. 19."""
        rho, u, p = P[0], P[1:4], P[4]
        lor = np.sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2])
        h = self.enthalpy(rho, p)
        U = np.empty_like(P)
        U[0] = lor * rho
        U[1:4] = lor * rho * h * u           # Gamma^2 rho h v with v = u / Gamma
        U[4] = lor * lor * rho * h - p - lor * rho
        return U

    def aux_from_prim(self, P):
        """Auxiliaries of Eq. 20: xi = Gamma^2 rho h and Gamma."""
        rho, u, p = P[0], P[1:4], P[4]
        lor = np.sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2])
        A = np.empty((2,) + P.shape[1:])
        A[0] = lor * lor * rho * self.enthalpy(rho, p)
        A[1] = lor
        return A

    def _pressure(self, xi, D, w, lor):
        """p(xi) and dp/dxi at fixed (D, S), with v^2 = w = S^2/xi^2, Gamma = lor and
        rho = D / Gamma (so d rho/d xi = D Gamma w / xi, and h = xi / (D Gamma) has
        dh/dxi = Gamma / D)."""
        ig2 = 1.0 - w
        rho = D / lor
        drho = D * lor * w / xi
        if self.eos == "synge":
            h = xi / (D * lor)
            theta = self.theta_of_h(h)
            dtheta = (5.0 - 9.0 * h / np.sqrt(9.0 * h * h + 16.0)) / 8.0
            return rho * theta, theta * drho + dtheta
        gm = (self.gamma - 1.0) / self.gamma
        return gm * (xi * ig2 - rho), gm * (1.0 + w - drho)

    def cons2prim(self, U, aux=None):
        """Primitive recovery as a root find in xi = Gamma^2 rho h (Section 2.3.4).

        With E = tau + D and S = |m|: v^2 = S^2/xi^2, Gamma = (1 - v^2)^-1/2, rho = D/Gamma,
        h = xi / (Gamma^2 rho) and p = p(rho, h) from the EOS; energy gives
        f(xi) = xi - p(xi) - E = 0. The root lies in [E, k E] with k = gamma for the ideal
        gas (p <= (gamma-1)/gamma xi) and k = 4/3 for the approximate Synge gas (h >= 4
        theta, so p <= xi/4). Newton's method with the analytic derivative runs from the
        stored auxiliary xi (when it lies inside the bracket, else the bracket's midpoint);
        a step leaving the closed bracket is replaced by bisection. It stops when
        |dxi| <= 1e-14 xi, at most 50 iterations. Returns (P, A) and raises on failure.
        """
        D = U[0]
        m = U[1:4]
        S2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2]
        E = U[4] + D
        lo = E.copy()
        hi = (4.0 / 3.0 if self.eos == "synge" else self.gamma) * E
        if aux is not None:
            xi = np.where((aux[0] > lo) & (aux[0] < hi), aux[0], 0.5 * (lo + hi))
        else:
            xi = 0.5 * (lo + hi)
        done = np.zeros(D.shape, dtype=bool)
        for _ in range(self.max_iter):
            w = S2 / (xi * xi)                   # v^2
            lor = 1.0 / np.sqrt(1.0 - w)
            p, dp = self._pressure(xi, D, w, lor)
            f = xi - p - E
            df = 1.0 - dp
            lo = np.where(f < 0.0, xi, lo)
            hi = np.where(f < 0.0, hi, xi)
            xn = xi - f / df
            inside = (xn >= lo) & (xn <= hi)
            xn = np.where(inside, xn, 0.5 * (lo + hi))
            conv = np.abs(xn - xi) <= self.tol * xn
            xi = np.where(done, xi, xn)
            done = done | conv
            if done.all():
                break
        if not done.all():
            raise FloatingPointError("srhd con2prim did not converge")
        w = S2 / (xi * xi)
        lor = 1.0 / np.sqrt(1.0 - w)
        P = np.empty_like(U)
        P[0] = D / lor
        P[1:4] = m * (lor / xi)                  # u = Gamma v, v = m / xi
        P[4] = self._pressure(xi, D, w, lor)[0]
        A = np.empty((2,) + U.shape[1:])
        A[0] = xi
        A[1] = lor
        return P, A

    def flux(self, P, U, d):
        """Flux along d of Eqs. 15-17: D v_d, m v_d + p e_d, m_d - D v_d."""
        u, p = P[1:4], P[4]
        lor = np.sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2])
        vd = u[d] / lor
        F = np.empty_like(P)
        F[0] = U[0] * vd
        for i in range(3):
            F[1 + i] = U[1 + i] * vd
        F[1 + d] = F[1 + d] + p
        F[4] = U[1 + d] - U[0] * vd
        return F

    def lambdas(self, P, d):
        """Characteristic speeds along d: the relativistic sound-wave speeds of a fluid with
        velocity v and sound speed cs (cs^2 from the EOS)."""
        rho, u, p = P[0], P[1:4], P[4]
        lor2 = 1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]
        v2 = 1.0 - 1.0 / lor2
        vd = u[d] / np.sqrt(lor2)
        cs2 = self.sound_speed2(rho, p)
        cs = np.sqrt(cs2)
        den = 1.0 - v2 * cs2
        root = cs * np.sqrt((1.0 - v2) * (1.0 - v2 * cs2 - vd * vd * (1.0 - cs2)))
        return (vd * (1.0 - cs2) - root) / den, (vd * (1.0 - cs2) + root) / den


class FFHD:
    """Frozen-field hydrodynamics (Section 2.3.2, Eqs. 7-9 without gravity, heating and the
    heat flux): U = (rho, m_par = rho v_par, e = p/(gamma-1) + rho v_par^2 / 2) moving along
    a frozen unit field b = B/|B| that is carried as three more variables (b_x, b_y, b_z)
    which are never updated. P = (rho, v_par, p, b).

    Discretisation (the paper gives the equations only):
      * b is not reconstructed: the face value of b_d is the mean of the two cells' b_d;
      * the flux along d is b_d,face (rho v, rho v^2 + p, (e + p) v) for the two face
        states (TVDLF, the module's solver in Table 1); the b variables carry the flux
        b_d,face along d (and 0 along the other axes), so the divergence of their fluxes
        is the discrete div b of the same face values;
      * the source p div b of the m_par equation (Eq. 8) uses that discrete div b and the
        cell pressure, so a state at rest with uniform p stays at rest in any field;
      * reflecting walls negate b_n (v_n = v_par b_n then changes sign), not m_par.
    """

    name = "ffhd"
    nvar = 6
    naux = 0
    glm = False
    nrec = 3            # variables that are reconstructed (the rest is taken cell-constant)
    frozen_from = 3     # variables from this index on are never updated

    def __init__(self, gamma: float):
        self.gamma = float(gamma)

    def cons2prim(self, U, aux=None):
        g = self.gamma
        P = np.empty_like(U)
        rho = U[0]
        v = U[1] / rho
        P[0] = rho
        P[1] = v
        P[2] = (g - 1.0) * (U[2] - 0.5 * rho * v * v)
        P[3:6] = U[3:6]
        return P, None

    def prim2cons(self, P):
        g = self.gamma
        U = np.empty_like(P)
        U[0] = P[0]
        U[1] = P[0] * P[1]
        U[2] = P[2] / (g - 1.0) + 0.5 * P[0] * P[1] * P[1]
        U[3:6] = P[3:6]
        return U

    def interface(self, PL, PR, d):
        """Both face states carry the mean of the two cells' b_d."""
        bf = 0.5 * (PL[3 + d] + PR[3 + d])
        PL = PL.copy()
        PR = PR.copy()
        PL[3 + d] = bf
        PR[3 + d] = bf
        return PL, PR

    def flux(self, P, U, d):
        rho, v, p, b = P[0], P[1], P[2], P[3 + d]
        F = np.zeros_like(P)
        F[0] = rho * v * b
        F[1] = (rho * v * v + p) * b
        F[2] = (U[2] + p) * v * b
        F[3 + d] = b
        return F

    def lambdas(self, P, d):
        """Signal speeds along d: (v_par -+ c_s) b_d (the speeds along the field projected)."""
        c = np.sqrt(self.gamma * P[2] / P[0])
        b = P[3 + d]
        a = P[1] * b
        w = c * np.abs(b)
        return a - w, a + w

    def source(self, Pc, L):
        """Adds p div b to the m_par equation; L[3..5] holds -d_d b_face,d."""
        L = L.copy()
        L[1] = L[1] - Pc[2] * ((L[3] + L[4]) + L[5])
        return L

    def reflect_vars(self, d):
        return [3 + d]


class FFHDHTC(FFHD):
    """Frozen-field hydrodynamics with hyperbolic field-aligned thermal conduction (Section
    2.3.2, Eqs. 7-10 without gravity and heating): U = (rho, m_par, e, q_par, b_x, b_y, b_z),
    P = (rho, v_par, p, q_par, b). The heat flux q_par relaxes towards kappa_par b.grad T
    (Eq. 10) and carries energy along the field: the energy flux is ((e + p) v_par - q_par) b
    (Eq. 9).

    Readings (the paper gives the equations and the relaxation time only):
      * q_par is reconstructed like rho, v_par and p (PLM); Eq. 10 has no divergence term, so
        q_par has no face flux of its own and no numerical dissipation;
      * the target kappa_par b.grad T uses T = p / rho (code units), kappa_par = kappa0
        T^(5/2) and grad T by central differences of the stage state across the cell's face
        neighbours, b the cell's frozen field;
      * tau = max(4 dt, tau_reduced) with tau_reduced = 0, i.e. tau = 4 dt; the relaxation
        -(q_par - kappa_par b.grad T) / tau is a source of every RK stage;
      * the signal speeds (and so the CFL step) are those of FFHD.
    """

    name = "ffhd_htc"
    nvar = 7
    naux = 0
    glm = False
    nrec = 4
    frozen_from = 4
    noflux = 3          # q_par: no face flux

    def __init__(self, gamma: float, kappa0: float):
        self.gamma = float(gamma)
        self.kappa0 = float(kappa0)

    def cons2prim(self, U, aux=None):
        g = self.gamma
        P = np.empty_like(U)
        rho = U[0]
        v = U[1] / rho
        P[0] = rho
        P[1] = v
        P[2] = (g - 1.0) * (U[2] - 0.5 * rho * v * v)
        P[3:7] = U[3:7]
        return P, None

    def prim2cons(self, P):
        g = self.gamma
        U = np.empty_like(P)
        U[0] = P[0]
        U[1] = P[0] * P[1]
        U[2] = P[2] / (g - 1.0) + 0.5 * P[0] * P[1] * P[1]
        U[3:7] = P[3:7]
        return U

    def interface(self, PL, PR, d):
        bf = 0.5 * (PL[4 + d] + PR[4 + d])
        PL = PL.copy()
        PR = PR.copy()
        PL[4 + d] = bf
        PR[4 + d] = bf
        return PL, PR

    def flux(self, P, U, d):
        rho, v, p, q, b = P[0], P[1], P[2], P[3], P[4 + d]
        F = np.zeros_like(P)
        F[0] = rho * v * b
        F[1] = (rho * v * v + p) * b
        F[2] = ((U[2] + p) * v - q) * b
        F[4 + d] = b
        return F

    def lambdas(self, P, d):
        c = np.sqrt(self.gamma * P[2] / P[0])
        b = P[4 + d]
        a = P[1] * b
        w = c * np.abs(b)
        return a - w, a + w

    def source(self, Pc, L):
        """p div b for m_par; L[4..6] holds -d_d b_face,d. (The q_par relaxation needs the
        time step and is added by the solver from htc_target.)"""
        L = L.copy()
        L[1] = L[1] - Pc[2] * ((L[4] + L[5]) + L[6])
        return L

    def htc_target(self, P, dx):
        """kappa0 T^(5/2) b.grad T on the 16^3 interior of a block whose primitives P carry
        two ghost layers (face neighbours filled); central differences per axis."""
        T = P[2] / P[0]
        i = slice(2, 18)
        Tc = T[i, i, i]
        grad = ((T[i, i, 3:19] - T[i, i, 1:17]) / (2.0 * dx[0]),
                (T[i, 3:19, i] - T[i, 1:17, i]) / (2.0 * dx[1]),
                (T[3:19, i, i] - T[1:17, i, i]) / (2.0 * dx[2]))
        bgrad = P[4][i, i, i] * grad[0] + P[5][i, i, i] * grad[1] + P[6][i, i, i] * grad[2]
        return self.kappa0 * Tc * Tc * np.sqrt(Tc) * bgrad

    def reflect_vars(self, d):
        return [4 + d]


def make_physics(name: str, gamma: float, eos: str = "ideal", kappa0: float = 0.0):
    if name == "srhd":
        return SRHD(gamma, eos)
    if eos != "ideal":
        raise ValueError("the Synge EOS applies to srhd only")
    if name == "ffhd_htc":
        return FFHDHTC(gamma, kappa0)
    return {"hd": HD, "mhd": MHD, "ffhd": FFHD}[name](gamma)
