"""Plain FP64 CPU block-AMR finite-volume solver: the oracle for the CUDA path.

TEST INFRASTRUCTURE ONLY (tests, the smoke check and the bench's CPU-baseline leg).

The method is the one-substep update of the paper's Section 2.1.3 (macro-kernel: primitive
conversion, reconstruction, Riemann flux, flux divergence, stage update) driven by the time
loop of Fig. 2 (set dt, advance with ghost exchange, error estimate, refine/coarsen with
prolongation/restriction) on 16^3-cell blocks with 2 ghost layers (Section 3.1).
Where the paper names a method without its formula, this file follows the readings listed
in the design notes (limiters, Davis HLL speeds, Rusanov TVDLF speed, Shu-Osher SSPRK,
max-sum CFL dt, Strang-split GLM decay, face-ghost order, minmod prolongation, the
axis-only Loehner estimator, 2:1 balance over faces, edges and corners).

Storage is deliberately plain: every leaf block owns a (nvar+naux, 20, 20, 20) array in
(v, z, y, x) order with the 2 ghost layers included. Edge and corner ghost cells are set to
NaN: the face-based unsplit stencil, the estimator and the prolongation never read them,
and a NaN would expose any read.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .cooling import Cooling
from .physics import make_physics

NB = 16          # interior cells per block edge
G = 2            # ghost layers
NT = NB + 2 * G  # stored cells per block edge

PERIODIC, OUTFLOW, REFLECT = "periodic", "outflow", "reflect"

# SSPRK stage weights: U_new = a * U^n + b * (U_s + dt L(U_s)) (Shu & Osher 1988).
RK_STAGES = {
    2: ((0.0, 1.0), (0.5, 0.5)),
    3: ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0)),
}


@dataclass
class Config:
    physics: str = "hd"
    limiter: str = "minmod"        # 'minmod' | 'vanleer'
    flux: str = "hll"              # 'hll' | 'tvdlf' | 'hllc' (hd only)
    rk: int = 2
    gamma: float = 5.0 / 3.0
    eos: str = "ideal"             # srhd: 'ideal' (Eq. 21) | 'synge' (approximate Synge gas)
    cfl: float = 0.4
    glm_alpha: float = 0.5
    base_blocks: tuple = (4, 4, 4)
    xmin: tuple = (0.0, 0.0, 0.0)
    xmax: tuple = (1.0, 1.0, 1.0)
    bc: tuple = (PERIODIC,) * 6    # faces -x, +x, -y, +y, -z, +z
    max_level: int = 1
    refine_vars: tuple = (0,)
    refine_weights: tuple = (1.0,)
    refine_tol: float = 0.2
    derefine_ratio: float = 1.0 / 8.0
    lohner_eps: float = 0.01
    cooling: tuple = None          # (T, Lambda) table: optically thin losses (hd, mhd)
    htc_kappa0: float = 0.0        # ffhd_htc: kappa_par = htc_kappa0 T^(5/2)
    eta: float = 0.0               # mhd: uniform resistivity (Section 2.3.3)


def morton3(ix: int, iy: int, iz: int) -> int:
    """Morton (Z-order) key with x in the lowest bit of each triple."""
    m = 0
    for b in range(21):
        m |= ((ix >> b) & 1) << (3 * b)
        m |= ((iy >> b) & 1) << (3 * b + 1)
        m |= ((iz >> b) & 1) << (3 * b + 2)
    return m


def minmod(a, b):
    """minmod(a, b) = sgn(a) min(|a|, |b|) if a b > 0, else 0."""
    return np.where((a > 0) & (b > 0), np.minimum(a, b),
                    np.where((a < 0) & (b < 0), np.maximum(a, b), 0.0))


def vanleer(a, b):
    """van Leer (1974) harmonic limiter 2ab/(a+b) if a b > 0, else 0."""
    pos = ((a > 0) & (b > 0)) | ((a < 0) & (b < 0))
    den = np.where(pos, a + b, 1.0)
    return np.where(pos, 2.0 * a * b / den, 0.0)


def restrict8(F):
    """Mean of each 2x2x2 cell group of F[..., 2Z, 2Y, 2X] (equal volumes).

    The eight terms are added in a fixed order, x fastest, then y, then z.
    """
    def f(dz, dy, dx):
        return F[..., dz::2, dy::2, dx::2]
    s = f(0, 0, 0) + f(0, 0, 1)
    s = s + f(0, 1, 0)
    s = s + f(0, 1, 1)
    s = s + f(1, 0, 0)
    s = s + f(1, 0, 1)
    s = s + f(1, 1, 0)
    s = s + f(1, 1, 1)
    return s * 0.125


def _ax(d: int) -> int:
    """Block-array axis of physical dimension d for arrays shaped (v, z, y, x)."""
    return 3 - d


def _S(r):
    """Index tuple (all vars, z, y, x) from per-dimension slices r = [x, y, z]."""
    return (slice(None), r[2], r[1], r[0])


class Solver:
    """Oracle block-AMR solver with calls mirroring the C-ABI of the CUDA library."""

    def __init__(self, cfg: Config):
        self.cfg = cfg
        self.phys = make_physics(cfg.physics, cfg.gamma, cfg.eos, cfg.htc_kappa0)
        if cfg.physics in ("ffhd", "ffhd_htc") and cfg.max_level != 1:
            raise ValueError("ffhd runs on uniform meshes (max_level 1)")
        if cfg.eta < 0.0 or (cfg.eta > 0.0 and cfg.physics != "mhd"):
            raise ValueError("resistivity eta >= 0 applies to mhd")
        self.cool = None
        if cfg.cooling is not None:
            if cfg.physics not in ("hd", "mhd", "ffhd", "ffhd_htc"):
                raise ValueError("radiative losses apply to hd, mhd and ffhd")
            self.cool = Cooling(cfg.cooling[0], cfg.cooling[1], cfg.gamma)
        self.nvar = self.phys.nvar
        self.naux = self.phys.naux
        self.nv = self.nvar + self.naux
        self.periodic = [cfg.bc[2 * d] == PERIODIC for d in range(3)]
        for d in range(3):
            if (cfg.bc[2 * d] == PERIODIC) != (cfg.bc[2 * d + 1] == PERIODIC):
                raise ValueError("periodic boundaries must be set on both faces")
        self.leaves = {}   # key (lev, ix, iy, iz) -> array (nv, 20, 20, 20)
        for iz in range(cfg.base_blocks[2]):
            for iy in range(cfg.base_blocks[1]):
                for ix in range(cfg.base_blocks[0]):
                    self.leaves[(1, ix, iy, iz)] = self._new_block()
        self.t = 0.0
        self.ic = None

    # ------------------------------------------------------------------ geometry
    def _new_block(self):
        a = np.full((self.nv, NT, NT, NT), np.nan)
        return a

    def nblocks(self, lev):
        return [b << (lev - 1) for b in self.cfg.base_blocks]

    def dx(self, lev):
        """Cell size per dimension at level lev."""
        c = self.cfg
        return [(c.xmax[d] - c.xmin[d]) / (c.base_blocks[d] * NB * (1 << (lev - 1)))
                for d in range(3)]

    def cell_centres(self, key):
        lev, ix, iy, iz = key
        dx = self.dx(lev)
        c = self.cfg
        i = np.arange(NB) + 0.5
        x = c.xmin[0] + (ix * NB + i) * dx[0]
        y = c.xmin[1] + (iy * NB + i) * dx[1]
        z = c.xmin[2] + (iz * NB + i) * dx[2]
        Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
        return X.ravel(), Y.ravel(), Z.ravel()

    def wrap(self, lev, pos):
        """Block position at level lev, wrapped on periodic axes; None if outside."""
        n = self.nblocks(lev)
        out = list(pos)
        for d in range(3):
            if out[d] < 0 or out[d] >= n[d]:
                if not self.periodic[d]:
                    return None
                out[d] %= n[d]
        return tuple(out)

    def leaf_covering(self, lev, pos):
        """Leaf at level <= lev covering block position pos of level lev, or None if finer."""
        l, p = lev, tuple(pos)
        while l >= 1:
            if (l,) + p in self.leaves:
                return (l,) + p
            l -= 1
            p = tuple(q >> 1 for q in p)
        return None

    def face_kind(self, key, d, s):
        """Neighbour relation across face (d, s): ('bc',), ('same', k), ('coarser', k, n),
        ('finer', [k...]) -- the srl / c / f classes of the paper's ghost exchange."""
        lev = key[0]
        pos = list(key[1:])
        pos[d] += s
        n = self.wrap(lev, pos)
        if n is None:
            return ("bc",)
        if (lev,) + n in self.leaves:
            return ("same", (lev,) + n)
        if lev > 1 and (lev - 1,) + tuple(q >> 1 for q in n) in self.leaves:
            return ("coarser", (lev - 1,) + tuple(q >> 1 for q in n), n)
        kids = []
        for t2 in range(2):
            for t1 in range(2):
                o = [0, 0, 0]
                o[d] = 1 if s < 0 else 0
                tang = [e for e in range(3) if e != d]
                o[tang[0]] = t1
                o[tang[1]] = t2
                k = (lev + 1,) + tuple(2 * n[e] + o[e] for e in range(3))
                if k not in self.leaves:
                    raise RuntimeError("mesh is not 2:1 balanced at %r" % (key,))
                kids.append(k)
        return ("finer", kids)

    def ordered_keys(self):
        """Leaves by level, then Morton order within the level."""
        return sorted(self.leaves, key=lambda k: (k[0], morton3(k[1], k[2], k[3])))

    # ------------------------------------------------------------------ state I/O
    def _prim_to_block(self, prim):
        P = prim.reshape(self.nvar, NB, NB, NB)
        U = self.phys.prim2cons(P)
        blk = self._new_block()
        blk[(slice(0, self.nvar),) + (slice(G, G + NB),) * 3] = U
        if self.naux:
            blk[(slice(self.nvar, self.nv),) + (slice(G, G + NB),) * 3] = self.phys.aux_from_prim(P)
        return blk

    def set_state(self, ic):
        """Evaluate the primitive initial condition at cell centres of every leaf (Fig. 1)."""
        self.ic = ic
        for key in self.leaves:
            self.leaves[key] = self._prim_to_block(np.asarray(ic(*self.cell_centres(key))))

    def set_state_blocks(self, cons):
        """Set conserved interiors of the leaves in `ordered_keys` order; aux guesses zero."""
        keys = self.ordered_keys()
        cons = np.asarray(cons, dtype=np.float64).reshape(len(keys), self.nvar, NB, NB, NB)
        for i, key in enumerate(keys):
            blk = self._new_block()
            blk[(slice(0, self.nvar),) + (slice(G, G + NB),) * 3] = cons[i]
            if self.naux:
                blk[(slice(self.nvar, self.nv),) + (slice(G, G + NB),) * 3] = 0.0
            self.leaves[key] = blk

    def get_state(self):
        """(levels[nblk], ijk[nblk, 3], cons[nblk, nvar, 16, 16, 16]) in ordered_keys order."""
        keys = self.ordered_keys()
        lev = np.array([k[0] for k in keys], dtype=np.int32)
        ijk = np.array([k[1:] for k in keys], dtype=np.int32).reshape(-1, 3)
        cons = np.stack([self.leaves[k][(slice(0, self.nvar),) + (slice(G, G + NB),) * 3]
                         for k in keys]) if keys else np.zeros((0, self.nvar, NB, NB, NB))
        return lev, ijk, cons

    def get_aux(self):
        keys = self.ordered_keys()
        return np.stack([self.leaves[k][(slice(self.nvar, self.nv),) + (slice(G, G + NB),) * 3]
                         for k in keys])

    def conserved_sums(self):
        """Volume integrals of every conserved variable over the leaves (log diagnostics)."""
        tot = [[] for _ in range(self.nvar)]
        for key, blk in self.leaves.items():
            dx = self.dx(key[0])
            dv = dx[0] * dx[1] * dx[2]
            for v in range(self.nvar):
                tot[v].append(float(np.sum(blk[(v,) + (slice(G, G + NB),) * 3])) * dv)
        return np.array([math.fsum(t) for t in tot])

    # ------------------------------------------------------------------ ghost cells
    def _ghost_slab(self, d, s):
        """Per-dimension slices of the 2 face-ghost layers (d, s) over the face interior."""
        r = [slice(G, G + NB)] * 3
        r[d] = slice(0, G) if s < 0 else slice(G + NB, NT)
        return r

    def _apply_bc(self, blk, d, s):
        """Physical boundary ghosts: outflow copies the nearest interior cell; reflect
        mirrors the interior with the normal momentum (and normal B) negated."""
        kind = self.cfg.bc[2 * d + (1 if s > 0 else 0)]
        r = self._ghost_slab(d, s)
        if kind == OUTFLOW:
            src = [slice(G, G + NB)] * 3
            src[d] = slice(G, G + 1) if s < 0 else slice(G + NB - 1, G + NB)
            blk[_S(r)] = blk[_S(src)]          # broadcasts over both layers
            return
        if kind != REFLECT:
            raise ValueError(kind)
        for layer in range(G):
            dst = [slice(G, G + NB)] * 3
            src = [slice(G, G + NB)] * 3
            if s < 0:
                dst[d] = slice(G - 1 - layer, G - layer)        # -1, -2
                src[d] = slice(G + layer, G + layer + 1)        #  0,  1
            else:
                dst[d] = slice(G + NB + layer, G + NB + layer + 1)   # 16, 17
                src[d] = slice(G + NB - 1 - layer, G + NB - layer)   # 15, 14
            blk[_S(dst)] = blk[_S(src)]
            if hasattr(self.phys, "reflect_vars"):
                for v in self.phys.reflect_vars(d):
                    blk[(v,) + _S(dst)[1:]] *= -1.0
                continue
            blk[(1 + d,) + _S(dst)[1:]] *= -1.0
            if self.phys.name == "mhd":
                blk[(5 + d,) + _S(dst)[1:]] *= -1.0

    def _fill_same(self, blk, nbr, d, s):
        r = self._ghost_slab(d, s)
        src = [slice(G, G + NB)] * 3
        src[d] = slice(NB, NB + G) if s < 0 else slice(G, 2 * G)
        blk[_S(r)] = nbr[_S(src)]

    def _fill_restrict(self, blk, kids, d, s):
        """Coarse ghosts from 4 finer neighbours: mean of the 8 fine cells they cover."""
        tang = [e for e in range(3) if e != d]
        for idx, k in enumerate(kids):
            t1, t2 = idx & 1, idx >> 1
            fine = self.leaves[k]
            src = [slice(G, G + NB)] * 3
            src[d] = slice(G + NB - 2 * G, G + NB) if s < 0 else slice(G, G + 2 * G)
            coarse = restrict8(fine[_S(src)])
            dst = self._ghost_slab(d, s)
            dst[tang[0]] = slice(G + 8 * t1, G + 8 * t1 + 8)
            dst[tang[1]] = slice(G + 8 * t2, G + 8 * t2 + 8)
            blk[_S(dst)] = coarse

    def _coarse_slopes(self, ckey, cache):
        """Limited slopes of the coarse block's interior cells, one per dimension.

        sigma_d = minmod(u[c+e_d] - u[c], u[c] - u[c-e_d]) from the coarse block's interior
        and its face ghosts filled by same-level copy, restriction or physical boundary.
        Face ghosts that only prolongation from a still coarser block would fill are not
        available at this point; the slope is then zero in that dimension.
        """
        if ckey in cache:
            return cache[ckey]
        blk = self.leaves[ckey]
        sig = []
        for d in range(3):
            c = [slice(G, G + NB)] * 3
            p = [slice(G, G + NB)] * 3
            m = [slice(G, G + NB)] * 3
            p[d] = slice(G + 1, G + NB + 1)
            m[d] = slice(G - 1, G + NB - 1)
            uc = blk[_S(c)]
            dp = blk[_S(p)] - uc
            dm = uc - blk[_S(m)]
            sg = minmod(dp, dm)
            for s in (-1, 1):
                if self.face_kind(ckey, d, s)[0] == "coarser":
                    edge = [slice(None)] * 3
                    edge[d] = slice(0, 1) if s < 0 else slice(NB - 1, NB)
                    sg[_S(edge)] = 0.0
            sig.append(sg)
        cache[ckey] = (blk[(slice(None),) + (slice(G, G + NB),) * 3], sig)
        return cache[ckey]

    @staticmethod
    def _prolong_cells(uc, sig, cidx, sgn):
        """u_f = u_C + 1/4 ((s_x sigma_x + s_y sigma_y) + s_z sigma_z) for fine cells f with
        parent-cell indices cidx (arrays per dimension) and child offsets sgn (+/-1)."""
        ii = (slice(None), cidx[2], cidx[1], cidx[0])
        acc = sgn[0] * sig[0][ii] + sgn[1] * sig[1][ii]
        acc = acc + sgn[2] * sig[2][ii]
        return uc[ii] + 0.25 * acc

    def _fill_prolong(self, blk, key, d, s, ckey, npos, cache):
        """Fine ghosts from the coarser neighbour ckey by limited-linear prolongation.

        The ghost cells lie in block position npos (level of key); in npos-local fine
        indices f they sit in coarse cell c = 8 (npos mod 2) + f // 2, at the child offset
        -1/4 (f even) or +1/4 (f odd) of the coarse cell size.
        """
        uc, sig = self._coarse_slopes(ckey, cache)
        r = self._ghost_slab(d, s)
        loc = []
        for e in range(3):
            if e == d:
                f = np.arange(NB - G, NB) if s < 0 else np.arange(0, G)
            else:
                f = np.arange(NB)
            loc.append(f)
        FZ, FY, FX = np.meshgrid(loc[2], loc[1], loc[0], indexing="ij")
        f3 = (FX, FY, FZ)
        cidx = [8 * (npos[e] & 1) + f3[e] // 2 for e in range(3)]
        sgn = [np.where(f3[e] % 2 == 0, -1.0, 1.0) for e in range(3)]
        blk[_S(r)] = self._prolong_cells(uc, sig, cidx, sgn)

    def fill_ghosts(self):
        """Face-ghost fill of every leaf: same-level copy, restriction and physical BCs
        first, then prolongation from coarser neighbours (the srl / f / c classes)."""
        later = []
        for key, blk in self.leaves.items():
            for d in range(3):
                for s in (-1, 1):
                    fk = self.face_kind(key, d, s)
                    if fk[0] == "same":
                        self._fill_same(blk, self.leaves[fk[1]], d, s)
                    elif fk[0] == "bc":
                        self._apply_bc(blk, d, s)
                    elif fk[0] == "finer":
                        self._fill_restrict(blk, fk[1], d, s)
                    else:
                        later.append((key, d, s, fk[1], fk[2]))
        cache = {}
        for key, d, s, ckey, npos in later:
            self._fill_prolong(self.leaves[key], key, d, s, ckey, npos, cache)

    # ------------------------------------------------------------------ the update
    def _prims(self, blk):
        """Primitives on interior + face ghosts (edge/corner cells stay NaN)."""
        U = blk[:self.nvar]
        aux = blk[self.nvar:] if self.naux else None
        if self.phys.name != "srhd":
            return self.phys.cons2prim(U)[0], None
        P = np.full(U.shape, np.nan)
        A = np.full((2,) + U.shape[1:], np.nan)
        regions = [(slice(G, G + NB),) * 3]
        for d in range(3):
            r = [slice(G, G + NB)] * 3
            r[d] = slice(0, NT)
            regions.append(tuple(r[::-1]))
        for reg in regions:
            idx = (slice(None),) + reg
            p, a = self.phys.cons2prim(U[idx], aux[idx])
            P[idx] = p
            A[idx] = a
        return P, A

    def _face_fluxes(self, P, d, dxl, ch):
        """Fluxes on the 17 faces along d of the 16x16 face columns of one block.

        PLM on primitives: P_L = P_i + sigma_i / 2, P_R = P_{i+1} - sigma_{i+1} / 2 with
        sigma_i = phi(P_i - P_{i-1}, P_{i+1} - P_i); then HLL (Davis speeds) or TVDLF.
        Returns an array (nvar, ...) with the face axis in place of dimension d.
        """
        phys = self.phys
        lim = minmod if self.cfg.limiter == "minmod" else vanleer
        r = [slice(G, G + NB)] * 3
        r[d] = slice(0, NT)
        Pd = np.moveaxis(P[_S(r)], _ax(d), -1)         # (nvar, a, b, 20)
        dl = Pd[..., 1:NT - 1] - Pd[..., 0:NT - 2]
        dr = Pd[..., 2:NT] - Pd[..., 1:NT - 1]
        sig = lim(dl, dr)                                # cells 1..18
        nrec = getattr(phys, "nrec", phys.nvar)
        sig[nrec:] = 0.0                                 # cell-constant variables (ffhd b)
        PL = Pd[..., 1:NT - 2] + 0.5 * sig[..., 0:NT - 3]
        PR = Pd[..., 2:NT - 1] - 0.5 * sig[..., 1:NT - 2]
        if phys.glm:
            PL, PR = phys.glm_interface(PL, PR, d, ch)
        if hasattr(phys, "interface"):
            PL, PR = phys.interface(PL, PR, d)
        UL = phys.prim2cons(PL)
        UR = phys.prim2cons(PR)
        if phys.glm:
            FL = phys.flux(PL, UL, d, ch)
            FR = phys.flux(PR, UR, d, ch)
        else:
            FL = phys.flux(PL, UL, d)
            FR = phys.flux(PR, UR, d)
        lml, lpl = phys.lambdas(PL, d)
        lmr, lpr = phys.lambdas(PR, d)
        if self.cfg.flux == "tvdlf":
            c = np.maximum(np.maximum(np.abs(lml), np.abs(lpl)),
                           np.maximum(np.abs(lmr), np.abs(lpr)))
            F = 0.5 * (FL + FR) - 0.5 * c * (UR - UL)
        elif self.cfg.flux == "hllc":
            F = self._hllc(PL, PR, UL, UR, FL, FR, np.minimum(lml, lmr), np.maximum(lpl, lpr), d)
        else:
            sl = np.minimum(lml, lmr)
            sr = np.maximum(lpl, lpr)
            mid = (sr * FL - sl * FR + sl * sr * (UR - UL)) / (sr - sl)
            F = np.where(sl >= 0.0, FL, np.where(sr <= 0.0, FR, mid))
        if hasattr(phys, "frozen_from"):
            # frozen variables: their exact flux (equal on both sides), no dissipation
            F[phys.frozen_from:] = FL[phys.frozen_from:]
        if hasattr(phys, "noflux"):
            F[phys.noflux] = 0.0                         # a variable without a flux term
        return np.moveaxis(F, -1, _ax(d))

    def _hllc(self, PL, PR, UL, UR, FL, FR, sl, sr, d):
        """HLLC flux for hydrodynamics (Toro, Spruce & Speares 1994; Toro 2009, ch. 10):
        the HLL fan with the contact restored. Contact speed
        S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R))
             / (rho_L (S_L - u_L) - rho_R (S_R - u_R)),
        star states U*_K = rho_K (S_K - u_K)/(S_K - S*) [1, S* e_d + v_t, E_K/rho_K +
        (S* - u_K)(S* + p_K / (rho_K (S_K - u_K)))], flux F_K + S_K (U*_K - U_K) on the side
        of the contact that contains x/t = 0."""
        if self.phys.name != "hd":
            raise ValueError("HLLC is available for hydrodynamics only (paper Table 1)")
        rl, rr = PL[0], PR[0]
        ul, ur = PL[1 + d], PR[1 + d]
        pl, pr = PL[4], PR[4]
        ss = (pr - pl + rl * ul * (sl - ul) - rr * ur * (sr - ur)) / (rl * (sl - ul) - rr * (sr - ur))

        def star(P, U, s):
            r, u, p = P[0], P[1 + d], P[4]
            fac = r * (s - u) / (s - ss)
            Us = np.empty_like(U)
            Us[0] = fac
            for i in range(3):
                Us[1 + i] = fac * P[1 + i]
            Us[1 + d] = fac * ss
            Us[4] = fac * (U[4] / r + (ss - u) * (ss + p / (r * (s - u))))
            return Us
        FsL = FL + sl * (star(PL, UL, sl) - UL)
        FsR = FR + sr * (star(PR, UR, sr) - UR)
        return np.where(sl >= 0.0, FL, np.where(ss >= 0.0, FsL, np.where(sr > 0.0, FsR, FR)))

    def _all_fluxes(self, ch):
        fluxes = {}
        new_aux = {}
        self._pcell = {}
        self._htc = {}
        for key, blk in self.leaves.items():
            P, A = self._prims(blk)
            if A is not None:
                new_aux[key] = A[(slice(None),) + (slice(G, G + NB),) * 3]
            if hasattr(self.phys, "source"):
                self._pcell[key] = P[(slice(None),) + (slice(G, G + NB),) * 3]
            dxl = self.dx(key[0])
            if hasattr(self.phys, "htc_target"):
                self._htc[key] = self.phys.htc_target(P, dxl)
            fluxes[key] = [self._face_fluxes(P, d, dxl, ch) for d in range(3)]
        return fluxes, new_aux

    @staticmethod
    def _face_of(F, d, idx):
        """Slice of a face-flux array F (nvar, z, y, x with faces along d) at face idx."""
        r = [slice(None)] * 3
        r[d] = slice(idx, idx + 1)
        return F[_S(r)]

    def _fixup(self, fluxes):
        """Coarse-fine flux correction: at every face a coarse block shares with 4 finer
        blocks, the coarse face flux is replaced by the mean of the 2x2 fine face fluxes
        (x-fastest order over the face's two tangential dimensions)."""
        for key in self.leaves:
            for d in range(3):
                for s in (-1, 1):
                    fk = self.face_kind(key, d, s)
                    if fk[0] != "finer":
                        continue
                    tang = [e for e in range(3) if e != d]
                    Fc = fluxes[key][d]
                    for idx, k in enumerate(fk[1]):
                        t1, t2 = idx & 1, idx >> 1
                        Ff = self._face_of(fluxes[k][d], d, NB if s < 0 else 0)
                        # Ff has extent 1 along d and 16 x 16 tangential.
                        def q(a, b, Ff=Ff):
                            r = [slice(None)] * 3
                            r[tang[0]] = slice(a, None, 2)
                            r[tang[1]] = slice(b, None, 2)
                            return Ff[_S(r)]
                        avg = (((q(0, 0) + q(1, 0)) + q(0, 1)) + q(1, 1)) * 0.25
                        dst = [slice(None)] * 3
                        dst[d] = slice(0, 1) if s < 0 else slice(NB, NB + 1)
                        dst[tang[0]] = slice(8 * t1, 8 * t1 + 8)
                        dst[tang[1]] = slice(8 * t2, 8 * t2 + 8)
                        Fc[_S(dst)] = avg

    def _rhs(self, fluxes, key):
        """L(U) = -sum_d (F_{i+1/2} - F_{i-1/2}) / dx_d on the block interior."""
        dx = self.dx(key[0])
        Fx, Fy, Fz = fluxes[key]
        lx = (Fx[:, :, :, 1:] - Fx[:, :, :, :-1]) / dx[0]
        ly = (Fy[:, :, 1:, :] - Fy[:, :, :-1, :]) / dx[1]
        lz = (Fz[:, 1:, :, :] - Fz[:, :-1, :, :]) / dx[2]
        return -((lx + ly) + lz)

    def signal_speeds(self):
        """(c_max, max over cells of sum_d (|v_d| + c_d) / dx_d) over leaf interiors."""
        cmax = 0.0
        smax = 0.0
        for key, blk in self.leaves.items():
            U = blk[(slice(None),) + (slice(G, G + NB),) * 3]
            if self.naux:
                P, _ = self.phys.cons2prim(U[:self.nvar], U[self.nvar:])
            else:
                P, _ = self.phys.cons2prim(U)
            dx = self.dx(key[0])
            tot = None
            for d in range(3):
                lm, lp = self.phys.lambdas(P, d)
                sp = np.maximum(np.abs(lm), np.abs(lp))
                cmax = max(cmax, float(sp.max()))
                tot = sp / dx[d] if tot is None else tot + sp / dx[d]
            smax = max(smax, float(tot.max()))
        return cmax, smax

    def resistive_rate(self):
        """2 eta sum_d dx_d^-2 at the finest level in use: the forward-Euler stability bound
        of the resistive diffusion term (its 7-point Laplacian) is dt <= 1 / that."""
        if self.cfg.eta <= 0.0:
            return 0.0
        lev = max(k[0] for k in self.leaves)
        return 2.0 * self.cfg.eta * sum(1.0 / (h * h) for h in self.dx(lev))

    def cfl_dt(self):
        """Set dt (Fig. 2): dt = CFL / max_cells sum_d (|v_d| + c_d)/dx_d; with resistivity
        the same Courant number scales the diffusive bound: dt = CFL / max(that maximum,
        2 eta sum_d dx_d^-2)."""
        _, smax = self.signal_speeds()
        return self.cfg.cfl / max(smax, self.resistive_rate())

    def _glm_decay(self, dt, ch):
        """psi <- psi exp(-dt/2 c_h alpha_GLM / min_d dx_d) (one Strang half, Section 2.3.3)."""
        for key, blk in self.leaves.items():
            dxm = min(self.dx(key[0]))
            blk[(8,) + (slice(G, G + NB),) * 3] *= math.exp(-0.5 * dt * ch * self.cfg.glm_alpha / dxm)

    def _cool(self, dt):
        """Radiative losses over dt on every leaf interior (exact integration, Section 2.3.1)."""
        inner = (slice(0, self.nvar),) + (slice(G, G + NB),) * 3
        for blk in self.leaves.values():
            blk[inner] = self.cool.apply(self.phys, blk[inner], dt)

    def step(self, dt=None, ch=None):
        """One full SSPRK step of every leaf (ghost fill, update and fix-up per stage).

        dt and the GLM speed c_h default to the CFL step and c_max of this mesh's state;
        a caller evolving a sub-domain of a larger mesh passes the global values."""
        cmax, smax = self.signal_speeds()
        if dt is None or dt <= 0:
            dt = self.cfg.cfl / max(smax, self.resistive_rate())
        if ch is None:
            ch = cmax
        if self.phys.glm:
            self._glm_decay(dt, ch)
        if self.cool is not None:       # Strang split: half the losses before, half after
            self._cool(0.5 * dt)
        inner = (slice(G, G + NB),) * 3
        un = {k: b[(slice(0, self.nvar),) + inner].copy() for k, b in self.leaves.items()}
        for a, b in RK_STAGES[self.cfg.rk]:
            self.fill_ghosts()
            fluxes, new_aux = self._all_fluxes(ch)
            self._fixup(fluxes)
            new = {}
            for key, blk in self.leaves.items():
                us = blk[(slice(0, self.nvar),) + inner]
                rhs = self._rhs(fluxes, key)
                if hasattr(self.phys, "source"):
                    rhs = self.phys.source(self._pcell[key], rhs)
                if self.cfg.eta > 0.0:
                    # resistive sources from the stage state with its face ghosts
                    sb, se = self.phys.resistive_source(blk[5:8], self.dx(key[0]), self.cfg.eta)
                    rhs[5:8] = rhs[5:8] + sb
                    rhs[4] = rhs[4] + se
                if hasattr(self.phys, "htc_target"):
                    # relaxation of q_par towards its target over tau = 4 dt (Eq. 10)
                    rhs[3] = -(us[3] - self._htc[key]) / (4.0 * dt)
                upd = us + dt * rhs
                if a != 0.0:
                    upd = a * un[key] + b * upd
                if hasattr(self.phys, "frozen_from"):
                    upd[self.phys.frozen_from:] = us[self.phys.frozen_from:]
                new[key] = upd
            for key, blk in self.leaves.items():
                blk[(slice(0, self.nvar),) + inner] = new[key]
                if self.naux:
                    blk[(slice(self.nvar, self.nv),) + inner] = new_aux[key]
        if self.phys.glm:
            self._glm_decay(dt, ch)
        if self.cool is not None:
            self._cool(0.5 * dt)
        self.t += dt
        return dt

    # ------------------------------------------------------------------ AMR
    def estimate(self):
        """Loehner error estimate per leaf: returns {key: max over interior cells of E}.

        Per variable u (weight w): E_u = sqrt(sum_d (u+ - 2 u0 + u-)^2 /
        sum_d (|u+ - u0| + |u0 - u-| + eps (|u+| + 2|u0| + |u-|))^2) with u+/- the
        neighbours along d; E = sum_u w E_u. FP64, every operation rounded separately in
        the order written (no fused multiply-add), so flags are reproducible bit for bit.
        """
        self.fill_ghosts()
        eps = self.cfg.lohner_eps
        out = {}
        for key, blk in self.leaves.items():
            etot = None
            for iv, w in zip(self.cfg.refine_vars, self.cfg.refine_weights):
                u = blk[iv]
                num = None
                den = None
                for d in range(3):
                    c = [slice(G, G + NB)] * 3
                    p = list(c)
                    m = list(c)
                    p[d] = slice(G + 1, G + NB + 1)
                    m[d] = slice(G - 1, G + NB - 1)
                    u0 = u[tuple(c[::-1])]
                    up = u[tuple(p[::-1])]
                    um = u[tuple(m[::-1])]
                    t = (up - 2.0 * u0) + um
                    q = (np.abs(up - u0) + np.abs(u0 - um)) + eps * ((np.abs(up) + 2.0 * np.abs(u0)) + np.abs(um))
                    num = t * t if num is None else num + t * t
                    den = q * q if den is None else den + q * q
                with np.errstate(invalid="ignore", divide="ignore"):
                    e = np.where(den > 0.0, np.sqrt(num / np.where(den > 0.0, den, 1.0)), 0.0)
                e = w * e
                etot = e if etot is None else etot + e
            out[key] = float(etot.max())
        return out

    def flags(self):
        """Per-leaf flags in ordered_keys order: +1 refine, -1 coarsen candidate, 0 keep."""
        est = self.estimate()
        c = self.cfg
        fl = {}
        for key, e in est.items():
            if e > c.refine_tol and key[0] < c.max_level:
                fl[key] = 1
            elif e < c.refine_tol * c.derefine_ratio and key[0] > 1:
                fl[key] = -1
            else:
                fl[key] = 0
        return fl, est

    def _dirs26(self):
        return [(a, b, c) for c in (-1, 0, 1) for b in (-1, 0, 1) for a in (-1, 0, 1)
                if (a, b, c) != (0, 0, 0)]

    def regrid(self, init=False):
        """Refine / coarsen the leaves from the estimator flags with 2:1 balance (Fig. 2).

        Refinement: flagged leaves below max_level, closed under 'a refined leaf's
        neighbours (faces, edges, corners) at a lower level refine too'. Coarsening: a
        parent whose 8 children are leaves, all flagged for coarsening and none refined,
        provided no block adjacent to the parent is refined in the post-refinement tree.
        New children are prolonged (limited linear, minmod) from the ghost-filled parent;
        a new parent is the mean of its 8 children. With init=True the initial condition
        is evaluated on every new block instead (Fig. 1).
        Returns (n_refined, n_coarsened) counted in parents.
        """
        fl, _ = self.flags()          # also fills ghosts (both phases)
        dirs = self._dirs26()
        R = {k for k, f in fl.items() if f == 1 and k[0] < self.cfg.max_level}
        changed = True
        while changed:
            changed = False
            for key in list(R):
                lev = key[0]
                for dv in dirs:
                    n = self.wrap(lev, (key[1] + dv[0], key[2] + dv[1], key[3] + dv[2]))
                    if n is None:
                        continue
                    leaf = self.leaf_covering(lev, n)
                    if leaf is not None and leaf[0] < lev and leaf not in R:
                        R.add(leaf)
                        changed = True
        internal = set()
        for key in self.leaves:
            lev, p = key[0], key[1:]
            while lev > 1:
                lev -= 1
                p = tuple(q >> 1 for q in p)
                internal.add((lev,) + p)
        internal |= R
        parents = {}
        for key in self.leaves:
            if key[0] > 1:
                pk = (key[0] - 1,) + tuple(q >> 1 for q in key[1:])
                parents.setdefault(pk, []).append(key)
        C = []
        for pk, kids in parents.items():
            if len(kids) != 8:
                continue
            if any(fl[k] != -1 or k in R for k in kids):
                continue
            ok = True
            lev = pk[0] + 1
            for k in kids:
                for dv in dirs:
                    n = self.wrap(lev, (k[1] + dv[0], k[2] + dv[1], k[3] + dv[2]))
                    if n is None or tuple(q >> 1 for q in n) == pk[1:]:
                        continue
                    if (lev,) + n in internal:
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                C.append(pk)
        # Apply: children of refined leaves, then coarsened parents.
        inner = (slice(G, G + NB),) * 3
        new_leaves = dict(self.leaves)
        for key in R:
            blk = self.leaves[key]
            del new_leaves[key]
            fine = self._prolong_block(key, blk)
            for o in range(8):
                ox, oy, oz = o & 1, (o >> 1) & 1, o >> 2
                ck = (key[0] + 1, 2 * key[1] + ox, 2 * key[2] + oy, 2 * key[3] + oz)
                cb = self._new_block()
                cb[(slice(None),) + inner] = fine[:, 16 * oz:16 * oz + 16, 16 * oy:16 * oy + 16,
                                                  16 * ox:16 * ox + 16]
                new_leaves[ck] = cb
        for pk in C:
            fine = np.empty((self.nv, 2 * NB, 2 * NB, 2 * NB))
            for o in range(8):
                ox, oy, oz = o & 1, (o >> 1) & 1, o >> 2
                ck = (pk[0] + 1, 2 * pk[1] + ox, 2 * pk[2] + oy, 2 * pk[3] + oz)
                fine[:, 16 * oz:16 * oz + 16, 16 * oy:16 * oy + 16, 16 * ox:16 * ox + 16] = \
                    self.leaves[ck][(slice(None),) + inner]
                del new_leaves[ck]
            pb = self._new_block()
            pb[(slice(None),) + inner] = restrict8(fine)
            new_leaves[pk] = pb
        created = [k for k in new_leaves if k not in self.leaves]
        self.leaves = new_leaves
        if init and self.ic is not None:
            for key in created:
                self.leaves[key] = self._prim_to_block(np.asarray(self.ic(*self.cell_centres(key))))
        return len(R), len(C)

    def _prolong_block(self, key, blk):
        """All 32^3 children cells of a ghost-filled parent by limited-linear prolongation."""
        sig = []
        for d in range(3):
            c = [slice(G, G + NB)] * 3
            p = list(c)
            m = list(c)
            p[d] = slice(G + 1, G + NB + 1)
            m[d] = slice(G - 1, G + NB - 1)
            uc = blk[_S(c)]
            sig.append(minmod(blk[_S(p)] - uc, uc - blk[_S(m)]))
        uc = blk[(slice(None),) + (slice(G, G + NB),) * 3]
        f = np.arange(2 * NB)
        FZ, FY, FX = np.meshgrid(f, f, f, indexing="ij")
        f3 = (FX, FY, FZ)
        cidx = [f3[e] // 2 for e in range(3)]
        sgn = [np.where(f3[e] % 2 == 0, -1.0, 1.0) for e in range(3)]
        return self._prolong_cells(uc, sig, cidx, sgn)

    # ------------------------------------------------------------------ checks
    def check_balance(self):
        """True when every pair of touching leaves differs by at most one level."""
        for key in self.leaves:
            lev = key[0]
            for dv in self._dirs26():
                n = self.wrap(lev, (key[1] + dv[0], key[2] + dv[1], key[3] + dv[2]))
                if n is None:
                    continue
                leaf = self.leaf_covering(lev, n)
                if leaf is not None:
                    if lev - leaf[0] > 1:
                        return False
                else:
                    # finer: children of (lev, n) touching key must be leaves (level lev+1)
                    for o in range(8):
                        ck = (lev + 1,) + tuple(2 * n[e] + ((o >> e) & 1) for e in range(3))
                        if ck not in self.leaves and self.leaf_covering(lev + 1, ck[1:]) is None:
                            # a child that is itself refined: is it adjacent to key?
                            touch = all(
                                (ck[1 + e] >> 1) == n[e] and (
                                    dv[e] == 0 or (dv[e] > 0 and ((ck[1 + e] & 1) == 0)) or
                                    (dv[e] < 0 and ((ck[1 + e] & 1) == 1)))
                                for e in range(3))
                            if touch:
                                return False
        return True
