"""Oracle: optically thin radiative losses integrated exactly (Townsend 2009), as the paper's
Section 2.3.1 prescribes for the energy sink -n_e n_H Lambda(T) of Eq. 4.

TEST INFRASTRUCTURE ONLY (see the package header): tests, the smoke check and the bench's
CPU-baseline leg are the only users. Shares no code with the CUDA library.

In code units the sink is de/dt = -rho^2 Lambda(T) with T = p / rho at fixed rho and
momentum, so the internal energy rho T / (gamma - 1) obeys

    dT/dt = -(gamma - 1) rho Lambda(T),   i.e.   integral_{T_new}^{T} dT' / Lambda(T') = r,
    r = (gamma - 1) rho dt.

Lambda is given as a table (T_k, Lambda_k), k = 0..N-1, and is a power law between nodes,
Lambda(T) = Lambda_k (T / T_k)^alpha_k on [T_k, T_{k+1}] (the last segment continues above
T_{N-1}); there is no loss at or below T_0, which is the floor. The integral of 1/Lambda
has a closed form on each segment, so the exact T_new follows by consuming r segment by
segment downward from T: with e = 1 - alpha_k,

    integral_{T_k}^{t} dT'/Lambda = (T_k / Lambda_k) expm1(e ln(t / T_k)) / e,

and inside a segment, below its upper end t with r' of r left,

    T_new = t exp(log1p(-e q) / e),   q = r' Lambda(t) / t

(e -> 0 limits: (T_k/Lambda_k) ln(t/T_k) and t exp(-q)). This is Townsend's exact
integration with the evolution function referred to each segment's own upper end instead of
the table's top node: the same integral, but every quantity stays on the scale of the local
cooling time, so no digits are lost where 1/Lambda near the top of the table dominates.
"""
from __future__ import annotations

import numpy as np


def _em1_over(e, x):
    """(exp(e x) - 1) / e, and its limit x at e = 0."""
    e = np.asarray(e, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    safe = np.where(e != 0.0, e, 1.0)
    return np.where(e != 0.0, np.expm1(e * x) / safe, x)


def _l1p_over(e, q):
    """log(1 - e q) / e, and its limit -q at e = 0."""
    e = np.asarray(e, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    safe = np.where(e != 0.0, e, 1.0)
    return np.where(e != 0.0, np.log1p(-e * q) / safe, -q)


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
        self.e = 1.0 - self.alpha
        # integral of 1/Lambda over each whole segment
        self.W = T[:-1] / L[:-1] * _em1_over(self.e, np.log(T[1:] / T[:-1]))

    def segment(self, t):
        """Segment index of temperature t: k with T_k <= t < T_{k+1}, clamped to 0..N-2."""
        k = np.searchsorted(self.T, t, side="right") - 1
        return np.clip(k, 0, self.T.size - 2)

    def lam(self, t):
        """The power-law Lambda(t) (segment of t; the last segment continues above)."""
        k = self.segment(t)
        return self.L[k] * (t / self.T[k]) ** self.alpha[k]

    def integral_below(self, t):
        """integral from T_k up to t of dT'/Lambda, k the segment of t."""
        k = self.segment(t)
        return self.T[k] / self.L[k] * _em1_over(self.e[k], np.log(t / self.T[k]))

    def cool_temperature(self, rho, t, dt):
        """Temperature after dt of losses at fixed rho (no change at or below T_0)."""
        shape = np.shape(t)
        t = np.asarray(t, dtype=np.float64).ravel()
        rho = np.broadcast_to(np.asarray(rho, dtype=np.float64), shape).ravel()
        out = t.copy()
        act = np.flatnonzero(t > self.T[0])
        if act.size == 0:
            return out.reshape(shape)
        r = self.g1 * rho[act] * dt            # integral of dT/Lambda still to consume
        top = t[act].copy()                    # upper end of the current partial segment
        k = self.segment(top)
        avail = self.integral_below(top)       # integral from T_k up to `top`
        lam_t = self.lam(top) / top            # Lambda(top) / top
        res = np.empty(act.size)
        live = np.ones(act.size, dtype=bool)
        while np.any(live):
            inside = live & (r < avail)
            if np.any(inside):
                q = r[inside] * lam_t[inside]
                res[inside] = top[inside] * np.exp(_l1p_over(self.e[k[inside]], q))
                live &= ~inside
            down = live & (k == 0)             # every segment consumed: the floor
            res[down] = self.T[0]
            live &= ~down
            if not np.any(live):
                break
            r = np.where(live, r - avail, r)
            k = np.where(live, k - 1, k)
            top = np.where(live, self.T[k + 1], top)
            avail = np.where(live, self.W[k], avail)
            lam_t = np.where(live, self.L[k + 1] / self.T[k + 1], lam_t)
        out[act] = np.maximum(res, self.T[0])
        return out.reshape(shape)

    def apply(self, phys, U, dt):
        """Losses over dt on conserved HD / MHD / FFHD states U (nvar, ...): only e
        changes, by rho (T_new - T) / (gamma - 1)."""
        P, _ = phys.cons2prim(U)
        ie = 2 if phys.name in ("ffhd", "ffhd_htc") else 4      # index of e in U and of p in P
        rho = P[0]
        t = P[ie] / rho
        tn = self.cool_temperature(rho, t, dt)
        out = U.copy()
        out[ie] = U[ie] - rho * (t - tn) / self.g1
        return out
