"""Thin Python binding of libagile.so (ctypes): argument marshalling only.

Every numerical step runs in the library's CUDA kernels. PyTorch supplies device memory
(its caching allocator, injected through agile_allocator) and the CUDA stream. There is no
fallback: if the compiled library is missing, loading raises.

The functions keep the C names (agile_mesh_create, agile_set_state, agile_cfl_dt,
agile_step, agile_regrid, agile_get_state, ...); `Mesh` wraps one mesh handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libagile.so")
NCELL = 4096

PHYSICS = {"hd": 0, "mhd": 1, "srhd": 2, "ffhd": 3, "ffhd_htc": 4}
NVAR = {0: 5, 1: 9, 2: 5, 3: 6, 4: 7}
EOS = {"ideal": 0, "synge": 1}
LIMITER = {"minmod": 0, "vanleer": 1}
FLUX = {"tvdlf": 0, "hll": 1, "hllc": 2}
BC = {"periodic": 0, "outflow": 1, "reflect": 2}
STATUS = {0: "AGILE_OK", 1: "AGILE_EINVAL", 2: "AGILE_ENOMEM", 3: "AGILE_EBUDGET",
          4: "AGILE_ECUDA", 5: "AGILE_ENOCONV", 6: "AGILE_EUNPHYS", 7: "AGILE_ETIMEOUT"}

# Symbols declared in include/agile.h (checked by the CPU test suite).
EXPORTS = ["agile_mesh_create", "agile_mesh_destroy", "agile_set_state", "agile_set_state_blocks",
           "agile_set_state_prims", "agile_batch_set_state_prims",
           "agile_cfl_dt", "agile_max_speeds", "agile_step", "agile_regrid", "agile_regrid_flags", "agile_get_layout",
           "agile_get_state", "agile_get_aux", "agile_conserved_sums",
           "agile_conserved_sums_noalloc", "agile_set_cooling", "agile_estimate",
           "agile_get_halo", "agile_sync", "agile_set_kernel_timing", "agile_kernel_timing",
           "agile_phase_timing",
           "agile_selftest_bounded_wait", "agile_selftest_rcp64", "agile_last_error", "agile_version",
           "agile_batch_create", "agile_batch_destroy", "agile_batch_layout",
           "agile_batch_set_state", "agile_batch_step", "agile_batch_cfl_dt", "agile_batch_copy_solve",
           "agile_batch_autotune", "agile_batch_regrid", "agile_batch_regrid_flags",
           "agile_batch_get_state", "agile_batch_sync", "agile_batch_launches",
           "agile_batch_attach", "agile_batch_detach",
           "agile_batch_last_error"]


class agile_config(C.Structure):
    _fields_ = [("physics", C.c_int), ("limiter", C.c_int), ("flux", C.c_int), ("rk", C.c_int),
                ("real_bytes", C.c_int), ("gamma", C.c_double), ("cfl", C.c_double),
                ("glm_alpha", C.c_double), ("base_blocks", C.c_int * 3), ("xmin", C.c_double * 3),
                ("xmax", C.c_double * 3), ("bc", C.c_int * 6), ("max_level", C.c_int),
                ("refine_nvars", C.c_int), ("refine_vars", C.c_int * 9),
                ("refine_weights", C.c_double * 9), ("refine_tol", C.c_double),
                ("derefine_ratio", C.c_double), ("lohner_eps", C.c_double), ("eos", C.c_int),
                ("htc_kappa0", C.c_double), ("eta", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
IC_FN = C.CFUNCTYPE(None, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                    C.c_int, C.POINTER(C.c_double), C.c_void_p)


class agile_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class AgileError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libagile.so (build it first with paper_2607_19277_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libagile.so not built at %s; run paper_2607_19277_gb300.build.build()" % path)
    lib = C.CDLL(path)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    sig = {
        "agile_mesh_create": (C.c_int, [C.POINTER(agile_config), C.POINTER(agile_allocator), P, C.POINTER(P)]),
        "agile_mesh_destroy": (None, [P]),
        "agile_set_state": (C.c_int, [P, IC_FN, P]),
        "agile_set_state_blocks": (C.c_int, [P, dp, C.c_size_t]),
        "agile_set_state_prims": (C.c_int, [P, dp, C.c_size_t]),
        "agile_batch_set_state_prims": (C.c_int, [P, C.c_int, dp, C.c_size_t]),
        "agile_cfl_dt": (C.c_int, [P, dp]),
        "agile_max_speeds": (C.c_int, [P, dp, dp]),
        "agile_step": (C.c_int, [P, C.c_double]),
        "agile_regrid": (C.c_int, [P, C.c_int, ip, ip]),
        "agile_regrid_flags": (C.c_int, [P, ip, C.c_int, ip, ip]),
        "agile_get_layout": (C.c_int, [P, C.POINTER(C.c_size_t), ip]),
        "agile_get_state": (C.c_int, [P, ip, ip, dp]),
        "agile_get_aux": (C.c_int, [P, dp]),
        "agile_conserved_sums": (C.c_int, [P, dp]),
        "agile_conserved_sums_noalloc": (C.c_int, [P, dp]),
        "agile_set_cooling": (C.c_int, [P, dp, dp, C.c_int]),
        "agile_estimate": (C.c_int, [P, dp]),
        "agile_get_halo": (C.c_int, [P, C.c_size_t, dp]),
        "agile_sync": (C.c_int, [P]),
        "agile_set_kernel_timing": (C.c_int, [P, C.c_int]),
        "agile_kernel_timing": (C.c_int, [P, dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "agile_phase_timing": (C.c_int, [P, dp, C.POINTER(C.c_longlong)]),
        "agile_selftest_bounded_wait": (C.c_int, [P, C.c_uint, ip]),
        "agile_selftest_rcp64": (C.c_int, [dp, dp, C.c_size_t, P, dp, dp]),
        "agile_last_error": (C.c_char_p, [P]),
        "agile_version": (C.c_char_p, []),
        "agile_batch_create": (C.c_int, [C.POINTER(agile_config), C.c_int, C.POINTER(agile_allocator), P, C.POINTER(P)]),
        "agile_batch_destroy": (None, [P]),
        "agile_batch_layout": (C.c_int, [P, C.c_int, C.POINTER(C.c_size_t), ip]),
        "agile_batch_set_state": (C.c_int, [P, C.c_int, IC_FN, P]),
        "agile_batch_step": (C.c_int, [P]),
        "agile_batch_cfl_dt": (C.c_int, [P, dp]),
        "agile_batch_get_state": (C.c_int, [P, C.c_int, ip, ip, dp]),
        "agile_batch_copy_solve": (C.c_int, [P, C.c_int, P, C.c_int]),
        "agile_batch_attach": (C.c_int, [P, C.POINTER(agile_config), ip]),
        "agile_batch_detach": (C.c_int, [P, C.c_int]),
        "agile_batch_autotune": (C.c_int, [P, C.c_int, ip, ip, ip, C.POINTER(C.c_float)]),
        "agile_batch_regrid": (C.c_int, [P, C.c_int, C.c_int, ip, ip]),
        "agile_batch_regrid_flags": (C.c_int, [P, C.c_int, ip, C.c_int, ip, ip]),
        "agile_batch_sync": (C.c_int, [P]),
        "agile_batch_launches": (C.c_longlong, [P]),
        "agile_batch_last_error": (C.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def make_config(physics="hd", limiter="minmod", flux="hll", rk=2, real_bytes=8, gamma=5.0 / 3.0,
                cfl=0.4, glm_alpha=0.5, base_blocks=(4, 4, 4), xmin=(0.0, 0.0, 0.0),
                xmax=(1.0, 1.0, 1.0), bc=("periodic",) * 6, max_level=1, refine_vars=(0,),
                refine_weights=(1.0,), refine_tol=0.2, derefine_ratio=1.0 / 8.0,
                lohner_eps=0.01, eos="ideal", htc_kappa0=0.0, eta=0.0) -> agile_config:
    c = agile_config()
    c.physics = PHYSICS[physics]
    c.limiter = LIMITER[limiter]
    c.flux = FLUX[flux]
    c.rk = rk
    c.real_bytes = real_bytes
    c.gamma = gamma
    c.cfl = cfl
    c.glm_alpha = glm_alpha
    for d in range(3):
        c.base_blocks[d] = base_blocks[d]
        c.xmin[d] = xmin[d]
        c.xmax[d] = xmax[d]
    for f in range(6):
        c.bc[f] = BC[bc[f]] if isinstance(bc[f], str) else bc[f]
    c.max_level = max_level
    c.refine_nvars = len(refine_vars)
    for i, (v, w) in enumerate(zip(refine_vars, refine_weights)):
        c.refine_vars[i] = v
        c.refine_weights[i] = w
    c.refine_tol = refine_tol
    c.derefine_ratio = derefine_ratio
    c.lohner_eps = lohner_eps
    c.eos = EOS[eos] if isinstance(eos, str) else eos
    c.htc_kappa0 = htc_kappa0
    c.eta = eta
    return c


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator on the mesh's stream."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device

        def alloc(nbytes, stream, ctx):
            try:
                return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, int(stream or 0))
            except Exception:
                return None

        def free(ptr, stream, ctx):
            if ptr:
                self.torch.cuda.caching_allocator_delete(int(ptr))

        self.c_alloc = ALLOC_FN(alloc)
        self.c_free = FREE_FN(free)
        self.struct = agile_allocator(self.c_alloc, self.c_free, None)


def check_rcp64(s, a):
    """Largest distance, in units of the last place of the IEEE quotient, and largest relative
    difference between the FP64 stencil's quotient of a by s (Newton-refined reciprocal
    estimate) and a / s, both formed on the device (agile_selftest_rcp64)."""
    lib = load()
    s = np.ascontiguousarray(s, dtype=np.float64).ravel()
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if s.shape != a.shape:
        raise ValueError("s and a differ in size")
    mu, mr = C.c_double(-1.0), C.c_double(-1.0)
    st = lib.agile_selftest_rcp64(_dptr(s), _dptr(a), s.size, None, C.byref(mu), C.byref(mr))
    _check(lib, None, st)
    return mu.value, mr.value


def _check(lib, mesh_ptr, st):
    if st != 0:
        msg = lib.agile_last_error(mesh_ptr) if mesh_ptr else b""
        raise AgileError(st, (msg or b"").decode())


def agile_mesh_create(cfg: agile_config, allocator=None, stream: int = 0):
    lib = load()
    out = C.c_void_p()
    st = lib.agile_mesh_create(C.byref(cfg), C.byref(allocator) if allocator is not None else None,
                               C.c_void_p(stream), C.byref(out))
    _check(lib, None, st)
    return out


class Mesh:
    """One block-AMR mesh on the current CUDA device and stream (torch's allocator)."""

    def __init__(self, cfg: agile_config, stream=None, use_torch_allocator=True, allocator=None):
        """allocator: an agile_allocator to use instead of torch's caching allocator (the
        caller keeps its callbacks alive); use_torch_allocator=False with no allocator
        selects the library's cudaMallocAsync default."""
        import torch
        self.lib = load()
        self.cfg = cfg
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        if allocator is not None:
            self._alloc = None
            alloc_struct = allocator
        else:
            self._alloc = _TorchAllocator(torch.cuda.current_device()) if use_torch_allocator else None
            alloc_struct = self._alloc.struct if self._alloc else None
        self.ptr = agile_mesh_create(cfg, alloc_struct, int(stream.cuda_stream))
        self.nvar = NVAR[cfg.physics]
        self.naux = 2 if cfg.physics == 2 else 0
        self._ic = None

    def close(self):
        if self.ptr:
            self.lib.agile_mesh_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        _check(self.lib, self.ptr, st)

    # --- calls of the C ABI -------------------------------------------------------------
    def set_state(self, ic):
        """ic(x, y, z) -> prim[nvar, n] (numpy); evaluated per block on the host."""
        nvar = self.nvar

        def cb(x, y, z, n, prim, user):
            xs = np.ctypeslib.as_array(x, shape=(n,)).copy()
            ys = np.ctypeslib.as_array(y, shape=(n,)).copy()
            zs = np.ctypeslib.as_array(z, shape=(n,)).copy()
            out = np.ctypeslib.as_array(prim, shape=(nvar * n,))
            out[:] = np.asarray(ic(xs, ys, zs), dtype=np.float64).reshape(nvar * n)

        self._ic = IC_FN(cb)   # kept alive: the library calls it again at regrid(init=1)
        self._ck(self.lib.agile_set_state(self.ptr, self._ic, None))

    def set_state_blocks(self, cons):
        cons = np.ascontiguousarray(cons, dtype=np.float64)
        self._ck(self.lib.agile_set_state_blocks(self.ptr, _dptr(cons), cons.shape[0]))

    def set_state_prims(self, prim):
        """Primitive values prim[nblk, nvar, 16, 16, 16] in the mesh's block order (see
        level1_cell_centres), converted to conserved variables on the device."""
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        self._ic = None
        self._ck(self.lib.agile_set_state_prims(self.ptr, _dptr(prim), prim.shape[0]))

    def cfl_dt(self) -> float:
        dt = C.c_double()
        self._ck(self.lib.agile_cfl_dt(self.ptr, C.byref(dt)))
        return dt.value

    def max_speeds(self):
        """(max_cells sum_d s_d / dx_d, c_max) of the current state."""
        a, b = C.c_double(), C.c_double()
        self._ck(self.lib.agile_max_speeds(self.ptr, C.byref(a), C.byref(b)))
        return a.value, b.value

    def step(self, dt: float = 0.0):
        self._ck(self.lib.agile_step(self.ptr, float(dt)))

    def regrid(self, init=False):
        nr, nc = C.c_int(), C.c_int()
        self._ck(self.lib.agile_regrid(self.ptr, int(init), C.byref(nr), C.byref(nc)))
        return nr.value, nc.value

    def regrid_flags(self, flags, init=False):
        f = np.ascontiguousarray(flags, dtype=np.int32)
        nr, nc = C.c_int(), C.c_int()
        self._ck(self.lib.agile_regrid_flags(self.ptr, _iptr(f), int(init), C.byref(nr), C.byref(nc)))
        return nr.value, nc.value

    def layout(self):
        n = C.c_size_t()
        nv = C.c_int()
        self._ck(self.lib.agile_get_layout(self.ptr, C.byref(n), C.byref(nv)))
        return n.value, nv.value

    def get_state(self):
        n, nv = self.layout()
        lev = np.zeros(n, dtype=np.int32)
        ijk = np.zeros((n, 3), dtype=np.int32)
        cons = np.zeros((n, nv, 16, 16, 16))
        self._ck(self.lib.agile_get_state(self.ptr, _iptr(lev), _iptr(ijk), _dptr(cons)))
        return lev, ijk, cons

    def get_aux(self):
        n, _ = self.layout()
        aux = np.zeros((n, 2, 16, 16, 16))
        self._ck(self.lib.agile_get_aux(self.ptr, _dptr(aux)))
        return aux

    def conserved_sums(self):
        s = np.zeros(self.nvar)
        self._ck(self.lib.agile_conserved_sums(self.ptr, _dptr(s)))
        return s

    def conserved_sums_noalloc(self):
        """Same sums through the entry point that allocates no device memory."""
        s = np.zeros(self.nvar)
        self._ck(self.lib.agile_conserved_sums_noalloc(self.ptr, _dptr(s)))
        return s

    def set_cooling(self, T=None, Lambda=None):
        """Radiative losses from the table (T, Lambda) (None switches them off)."""
        if T is None:
            self._ck(self.lib.agile_set_cooling(self.ptr, None, None, 0))
            return
        t = np.ascontiguousarray(T, dtype=np.float64)
        lam = np.ascontiguousarray(Lambda, dtype=np.float64)
        if t.shape != lam.shape or t.ndim != 1:
            raise ValueError("T and Lambda must be 1-D arrays of the same length")
        self._ck(self.lib.agile_set_cooling(self.ptr, _dptr(t), _dptr(lam), int(t.size)))

    def estimate(self):
        n, _ = self.layout()
        e = np.zeros(n)
        self._ck(self.lib.agile_estimate(self.ptr, _dptr(e)))
        return e

    def get_halo(self, block):
        out = np.zeros((self.nvar + self.naux, 20, 20, 20))
        self._ck(self.lib.agile_get_halo(self.ptr, block, _dptr(out)))
        return out

    def sync(self):
        self._ck(self.lib.agile_sync(self.ptr))

    def set_kernel_timing(self, enable=True):
        self._ck(self.lib.agile_set_kernel_timing(self.ptr, int(enable)))

    def kernel_timing(self):
        ms = C.c_double()
        n = C.c_longlong()
        tot = C.c_longlong()
        self._ck(self.lib.agile_kernel_timing(self.ptr, C.byref(ms), C.byref(n), C.byref(tot)))
        return ms.value, n.value, tot.value

    def phase_timing(self):
        """Device ms and launches per phase since timing was enabled: a dict over 'stage',
        'ghost_fill', 'fixup', 'estimate'."""
        ms = (C.c_double * 4)()
        n = (C.c_longlong * 4)()
        self._ck(self.lib.agile_phase_timing(self.ptr, ms, n))
        names = ("stage", "ghost_fill", "fixup", "estimate")
        return {k: (ms[i], n[i]) for i, k in enumerate(names)}


def morton3(i, j, k):
    """Morton (Z-order) key of integer block coordinates, x in the lowest bit of each triple
    (the library's block order within a level); numpy arrays or ints."""
    i, j, k = (np.asarray(a, dtype=np.int64) for a in (i, j, k))
    key = np.zeros(np.broadcast(i, j, k).shape, dtype=np.int64)
    for b in range(21):
        key |= ((i >> b) & 1) << (3 * b)
        key |= ((j >> b) & 1) << (3 * b + 1)
        key |= ((k >> b) & 1) << (3 * b + 2)
    return key


def level1_cell_centres(cfg: agile_config):
    """Cell centres (x, y, z), each of shape (nblk, 16, 16, 16), of a mesh of level-1 blocks
    in the library's block order (Morton order of the block coordinates) with cells [z][y][x],
    computed as the library computes them, so that ic(x, y, z) here gives the primitives
    agile_set_state would ask the callback for."""
    nb = [int(cfg.base_blocks[d]) for d in range(3)]
    bk, bj, bi = np.meshgrid(np.arange(nb[2]), np.arange(nb[1]), np.arange(nb[0]), indexing="ij")
    bi, bj, bk = bi.ravel(), bj.ravel(), bk.ravel()
    order = np.argsort(morton3(bi, bj, bk), kind="stable")
    bi, bj, bk = bi[order], bj[order], bk[order]
    c = np.arange(16)
    out = []
    for d, bb in enumerate((bi, bj, bk)):
        dx = (cfg.xmax[d] - cfg.xmin[d]) / (float(nb[d]) * 16 * 1.0)
        idx = (bb[:, None] * 16 + c[None, :]).astype(np.float64) + 0.5      # (nblk, 16)
        v = cfg.xmin[d] + idx * dx
        shape = [len(bb), 1, 1, 1]
        shape[3 - d] = 16
        out.append(np.broadcast_to(v.reshape(shape), (len(bb), 16, 16, 16)))
    return out[0], out[1], out[2]


def prims_of(ic, cfg: agile_config, out=None):
    """ic evaluated once at every cell centre of a level-1 mesh: prim[nblk, nvar, 16, 16, 16]
    in block order (the argument of Mesh.set_state_prims), written into `out` when given (a
    C-contiguous float64 array of that shape, e.g. in page-locked memory)."""
    x, y, z = level1_cell_centres(cfg)
    nblk = x.shape[0]
    p = np.asarray(ic(x.ravel(), y.ravel(), z.ravel()), dtype=np.float64)
    nvar = p.shape[0]
    blocks = p.reshape(nvar, nblk, 16, 16, 16).transpose(1, 0, 2, 3, 4)
    if out is None:
        return np.ascontiguousarray(blocks)
    if out.shape != blocks.shape or out.dtype != np.float64 or not out.flags["C_CONTIGUOUS"]:
        raise ValueError("out must be a C-contiguous float64 array of shape %s" % (blocks.shape,))
    out[...] = blocks
    return out


def _ic_callback(ic, nvar):
    def cb(x, y, z, n, prim, user):
        xs = np.ctypeslib.as_array(x, shape=(n,)).copy()
        ys = np.ctypeslib.as_array(y, shape=(n,)).copy()
        zs = np.ctypeslib.as_array(z, shape=(n,)).copy()
        out = np.ctypeslib.as_array(prim, shape=(nvar * n,))
        out[:] = np.asarray(ic(xs, ys, zs), dtype=np.float64).reshape(nvar * n)
    return IC_FN(cb)


class Batch:
    """Independent solves advanced together (one launch per RK stage over the blocks of all
    levels of all of them, each step replayed from a CUDA graph); refined per solve or all
    at once with regrid / regrid_flags."""

    def __init__(self, cfgs, stream=None, use_torch_allocator=True):
        import torch
        self.lib = load()
        self.cfgs = list(cfgs)
        arr = (agile_config * len(self.cfgs))(*self.cfgs)
        self.stream = stream
        self._alloc = _TorchAllocator(torch.cuda.current_device()) if use_torch_allocator else None
        out = C.c_void_p()
        st = self.lib.agile_batch_create(arr, len(self.cfgs), self._alloc.struct if self._alloc else None,
                                         C.c_void_p(int(stream.cuda_stream) if stream is not None else 0),
                                         C.byref(out))
        _check(self.lib, None, st)
        self.ptr = out
        self.nvar = NVAR[self.cfgs[0].physics]
        self._ics = {}

    def _ck(self, st):
        if st != 0:
            msg = self.lib.agile_batch_last_error(self.ptr)
            raise AgileError(st, (msg or b"").decode())

    def close(self):
        if self.ptr:
            self.lib.agile_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self, solve):
        n = C.c_size_t()
        nv = C.c_int()
        self._ck(self.lib.agile_batch_layout(self.ptr, solve, C.byref(n), C.byref(nv)))
        return n.value, nv.value

    def set_state(self, solve, ic):
        cb = _ic_callback(ic, self.nvar)
        self._ics[solve] = cb
        self._ck(self.lib.agile_batch_set_state(self.ptr, solve, cb, None))

    def set_state_prims(self, solve, prim):
        prim = np.ascontiguousarray(prim, dtype=np.float64)
        self._ics.pop(solve, None)
        self._ck(self.lib.agile_batch_set_state_prims(self.ptr, solve, _dptr(prim), prim.shape[0]))

    def step(self):
        self._ck(self.lib.agile_batch_step(self.ptr))

    def cfl_dt(self):
        dt = np.zeros(len(self.cfgs))
        self._ck(self.lib.agile_batch_cfl_dt(self.ptr, _dptr(dt)))
        return dt

    def get_state(self, solve):
        n, nv = self.layout(solve)
        lev = np.zeros(n, dtype=np.int32)
        ijk = np.zeros((n, 3), dtype=np.int32)
        cons = np.zeros((n, nv, 16, 16, 16))
        self._ck(self.lib.agile_batch_get_state(self.ptr, solve, _iptr(lev), _iptr(ijk), _dptr(cons)))
        return lev, ijk, cons

    def regrid(self, solve=-1, init=False):
        """Estimate-driven refinement of one solve (every solve for -1, with one new layout of
        the pools); returns (n_refined, n_coarsened)."""
        nr, nc = C.c_int(), C.c_int()
        self._ck(self.lib.agile_batch_regrid(self.ptr, solve, int(init), C.byref(nr), C.byref(nc)))
        return nr.value, nc.value

    def regrid_flags(self, solve, flags, init=False):
        f = np.ascontiguousarray(flags, dtype=np.int32)
        nr, nc = C.c_int(), C.c_int()
        self._ck(self.lib.agile_batch_regrid_flags(self.ptr, solve, _iptr(f), int(init), C.byref(nr), C.byref(nc)))
        return nr.value, nc.value

    def autotune(self, trials=3):
        """Pick the fastest stage-launch shape; returns (grid, dynamic, ms per shape, layout)."""
        g, d, lay = C.c_int(), C.c_int(), C.c_int()
        ms = (C.c_float * 18)()     # the library writes eighteen values
        self._ck(self.lib.agile_batch_autotune(self.ptr, int(trials), C.byref(g), C.byref(d),
                                               C.byref(lay), ms))
        return g.value, bool(d.value), list(ms), lay.value

    def attach(self, cfg):
        """Add a solve with configuration cfg (the batch's scheme) to the running batch;
        returns its index. Set its state before the next step."""
        idx = C.c_int()
        self._ck(self.lib.agile_batch_attach(self.ptr, C.byref(cfg), C.byref(idx)))
        return idx.value

    def detach(self, solve):
        """Remove a solve from the batch (the others keep their places and states)."""
        self._ck(self.lib.agile_batch_detach(self.ptr, int(solve)))

    def copy_solve(self, solve, src, src_solve):
        """Device-to-device copy of solve src_solve of Batch src into solve `solve`."""
        self._ck(self.lib.agile_batch_copy_solve(self.ptr, solve, src.ptr, src_solve))

    def sync(self):
        self._ck(self.lib.agile_batch_sync(self.ptr))

    def launches(self):
        return int(self.lib.agile_batch_launches(self.ptr))
