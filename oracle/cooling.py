"""Oracle: optically thin radiative losses integrated exactly (Townsend 2009), as the paper's
Section 2.3.1 prescribes for the energy sink -n_e n_H Lambda(T) of Eq. 3.

TEST INFRASTRUCTURE ONLY (see the package header): tests, the smoke check and the bench's
CPU-baseline leg are the only users. Shares no code with the CUDA library.

In code units the sink is de/dt = -rho^2 Lambda(T) with T = p / rho at fixed rho and
momentum, so the internal energy rho T / (gamma - 1) obeys

    dT/dt = -(gamma - 1) rho Lambda(T).

Lambda is given as a table (T_k, Lambda_k), k = 0..N-1, and is a power law between nodes,
Lambda(T) = Lambda_k (T / T_k)^alpha_k on [T_k, T_{k+1}] (the last segment continues above
T_{N-1}); there is no loss below T_0, which acts as a floor. With the reference node
T_ref = T_{N-1} and the temporal evolution function

    Y(T) = (Lambda_ref / T_ref) * integral_T^T_ref dT' / Lambda(T'),

the ODE integrates to Y(T_new) = Y(T_old) + (Lambda_ref / T_ref) (gamma - 1) rho dt, and
Y has a closed form and a closed-form inverse on every power-law segment. With
e = 1 - alpha_k and C_k = (Lambda_ref / T_ref) T_k / Lambda_k, the integral over segment k
from T to T_{k+1} gives

    Y(T) = Y_{k+1} + C_k (T/T_k)^e ((T_{k+1}/T)^e - 1) / e,

and, with s = (y - Y_{k+1}) / C_k and B_k = (T_{k+1}/T_k)^e, the inverse

    T = T_{k+1} (1 - e s / B_k)^(1/e).

Both are written with expm1 / log1p so that they stay accurate as e -> 0 (alpha -> 1),
where they tend to the logarithmic forms Y_{k+1} + C_k ln(T_{k+1}/T) and T_{k+1} exp(-s).
"""
from __future__ import annotations

import numpy as np


class Cooling:
    def __init__(self, T, L, gamma: float):
        T = np.asarray(T, dtype=np.float64)
        L = np.asarray(L, dtype=np.float64)
        if T.ndim != 1 or T.size < 2 or T.size != L.size:
            raise ValueError("cooling table needs at least two (T, Lambda) nodes")
        if not (np.all(np.diff(T) > 0) and np.all(T > 0) and np.all(L > 0)):
            raise ValueError("cooling table: T increasing, T > 0 and Lambda > 0")
        self.T = T
        self.L = L
        self.g1 = float(gamma) - 1.0
        self.alpha = np.log(L[1:] / L[:-1]) / np.log(T[1:] / T[:-1])
        self.Tref = T[-1]
        self.Lref = L[-1]
        n = T.size
        self.Y = np.zeros(n)
        for k in range(n - 2, -1, -1):
            self.Y[k] = self.Y[k + 1] + self._seg_integral(k, T[k], T[k + 1])

    @staticmethod
    def _em1_over(e, x):
        """(exp(e x) - 1) / e, and its limit x at e = 0."""
        return np.expm1(e * x) / e if e != 0.0 else x

    @staticmethod
    def _l1p_over(e, z):
        """log(1 - e z) / e, and its limit -z at e = 0."""
        return np.log1p(-e * z) / e if e != 0.0 else -z

    def _c(self, k):
        return self.Lref / self.Tref * self.T[k] / self.L[k]

    def _seg_integral(self, k, ta, tb):
        """(Lambda_ref / T_ref) integral_ta^tb dT / Lambda(T) on the power law of segment k."""
        e = 1.0 - self.alpha[k]
        return self._c(k) * (ta / self.T[k]) ** e * self._em1_over(e, np.log(tb / ta))

    def segment(self, t):
        """Segment index of temperature t: k with T_k <= t < T_{k+1}, clamped to 0..N-2."""
        k = np.searchsorted(self.T, t, side="right") - 1
        return np.clip(k, 0, self.T.size - 2)

    def y_of_t(self, t):
        k = self.segment(t)
        out = np.empty_like(t)
        for kk in np.unique(k):
            m = k == kk
            out[m] = self.Y[kk + 1] + self._seg_integral(kk, t[m], self.T[kk + 1])
        return out

    def t_of_y(self, y):
        """Inverse of Y: the temperature whose evolution function is y (T_0 when y >= Y_0)."""
        out = np.empty_like(y)
        floor = y >= self.Y[0]
        out[floor] = self.T[0]
        rest = ~floor
        # Y decreases with T: segment k holds Y_{k+1} <= y <= Y_k (last segment above T_ref)
        k = np.searchsorted(-self.Y, -y[rest], side="left") - 1
        k = np.clip(k, 0, self.T.size - 2)
        yr = y[rest]
        res = np.empty_like(yr)
        for kk in np.unique(k):
            m = k == kk
            e = 1.0 - self.alpha[kk]
            sk = (yr[m] - self.Y[kk + 1]) / self._c(kk)
            bk = (self.T[kk + 1] / self.T[kk]) ** e
            res[m] = self.T[kk + 1] * np.exp(self._l1p_over(e, sk / bk))
        out[rest] = res
        return out

    def cool_temperature(self, rho, t, dt):
        """Temperature after dt of losses at fixed rho (no change at or below T_0)."""
        t = np.asarray(t, dtype=np.float64)
        rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), t.shape)
        out = t.copy()
        act = t > self.T[0]
        if np.any(act):
            y = self.y_of_t(t[act]) + self.Lref / self.Tref * self.g1 * rho[act] * dt
            out[act] = np.maximum(self.t_of_y(y), self.T[0])
        return out

    def apply(self, phys, U, dt):
        """Losses over dt on conserved HD / MHD states U (nvar, ...): only e changes, by
        rho (T_new - T) / (gamma - 1)."""
        P, _ = phys.cons2prim(U)
        rho = P[0]
        t = P[4] / rho
        tn = self.cool_temperature(rho, t, dt)
        out = U.copy()
        out[4] = U[4] - rho * (t - tn) / self.g1
        return out
