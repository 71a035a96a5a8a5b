"""CPU checks of the library's host octree (csrc/mesh.cpp) against the oracle's separate
tree code: identical leaf sets and order after random refine/coarsen flag sequences,
identical neighbour classes (same / coarser / finer / boundary) per face, 2:1 balance, and
consistent ghost-slot tables. Both sides are independent implementations."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import Config, Solver
from paper_2607_19277_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
BCMAP = {"periodic": 0, "outflow": 1, "reflect": 2}
KIND = {0: "same", 1: "bc", 2: "coarser", 3: "finer"}


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("shim") / "libmeshshim.so")
    src = [os.path.join(HERE, "mesh_shim.cpp"),
           os.path.join(ROOT, "paper_2607_19277_gb300", "csrc", "mesh.cpp")]
    subprocess.run([gxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-o", out] + src, check=True)
    lib = C.CDLL(out)
    lib.shim_create.restype = C.c_void_p
    lib.shim_create.argtypes = [C.POINTER(C.c_int), C.c_int, C.POINTER(C.c_int)]
    for name in ("shim_destroy", "shim_nblocks", "shim_blocks", "shim_regrid", "shim_balanced",
                 "shim_faces"):
        getattr(lib, name).argtypes = [C.c_void_p] + ([C.c_void_p] if name in
                                                      ("shim_blocks", "shim_regrid", "shim_faces") else [])
    return lib


def _host_blocks(lib, h):
    n = lib.shim_nblocks(h)
    a = np.zeros((n, 4), dtype=np.int32)
    lib.shim_blocks(h, a.ctypes.data)
    return [tuple(r) for r in a.tolist()]


def _forced(o, flags_by_key):
    orig = o.flags

    def f():
        fl, est = orig()
        for k in fl:
            fl[k] = flags_by_key.get(k, 0)
        return fl, est
    o.flags = f
    try:
        return o.regrid()
    finally:
        o.flags = orig


@pytest.mark.parametrize("seed,base,bc", [
    (1, (2, 2, 1), ("periodic",) * 6),
    (2, (3, 2, 2), ("outflow", "outflow", "periodic", "periodic", "reflect", "reflect")),
    (3, (1, 2, 3), ("reflect", "outflow", "outflow", "reflect", "periodic", "periodic")),
])
def test_host_mesh_matches_oracle_tree(shim, seed, base, bc):
    rng = np.random.default_rng(seed)
    cfg = Config(physics="hd", base_blocks=base, bc=bc, max_level=4)
    o = Solver(cfg)
    o.set_state(W.uniform_state([1, 0, 0, 0, 1]))
    bca = (C.c_int * 6)(*[BCMAP[b] for b in bc])
    h = shim.shim_create((C.c_int * 3)(*base), 4, bca)
    n_coarsened = 0
    try:
        for it in range(8):
            keys = o.ordered_keys()
            assert _host_blocks(shim, h) == keys
            # random flags: refine some, coarsen-candidate many; the last two rounds flag
            # every leaf for coarsening
            if it >= 6:
                fl = -np.ones(len(keys), dtype=np.int64)
            else:
                fl = rng.choice([-1, 0, 1], size=len(keys), p=[0.5, 0.3, 0.2] if it > 2 else [0.1, 0.5, 0.4])
            by_key = {k: int(v) for k, v in zip(keys, fl)}
            ro = _forced(o, by_key)
            fl32 = np.ascontiguousarray(fl, dtype=np.int32)   # kept alive across the call
            rh = shim.shim_regrid(h, fl32.ctypes.data)
            assert (rh >> 16, rh & 0xFFFF) == ro
            n_coarsened += ro[1]
            assert shim.shim_balanced(h) == 1 and o.check_balance()
        assert n_coarsened > 0
        keys = o.ordered_keys()
        assert _host_blocks(shim, h) == keys
        faces = np.zeros((len(keys), 6, 5), dtype=np.int32)
        nslots = shim.shim_faces(h, faces.ctypes.data)
        assert nslots >= 0
        idx = {k: i for i, k in enumerate(keys)}
        n_cf = 0
        for i, k in enumerate(keys):
            for f in range(6):
                fk = o.face_kind(k, f >> 1, -1 if f % 2 == 0 else 1)
                assert KIND[faces[i, f, 0]] == fk[0], (k, f)
                if fk[0] == "same":
                    assert faces[i, f, 1] == idx[fk[1]]
                elif fk[0] == "coarser":
                    assert faces[i, f, 1] == idx[fk[1]]
                    n_cf += 1
                elif fk[0] == "finer":
                    assert list(faces[i, f, 1:]) == [idx[q] for q in fk[1]]
                    n_cf += 1
        assert nslots == n_cf
    finally:
        shim.shim_destroy(h)


@pytest.mark.parametrize("base", [(3, 2, 4), (4, 4, 4), (1, 5, 2)])
def test_level1_cell_centres_follow_the_host_block_order(shim, base):
    """The binding's cell centres for set_state_prims follow the library's block order (the
    host octree's level-1 blocks) and its centre formula."""
    from paper_2607_19277_gb300 import agile
    h = shim.shim_create((C.c_int * 3)(*base), 1, (C.c_int * 6)(*([0] * 6)))
    blocks = _host_blocks(shim, h)
    shim.shim_destroy(h)
    cfg = agile.make_config(base_blocks=base, xmin=(-0.3, 0.1, 2.0), xmax=(0.7, 0.9, 5.0))
    x, y, z = agile.level1_cell_centres(cfg)
    assert x.shape == (len(blocks), 16, 16, 16)
    for b, (lev, i, j, k) in enumerate(blocks):
        assert lev == 1
        for arr, d, bc in ((x, 0, i), (y, 1, j), (z, 2, k)):
            dx = (cfg.xmax[d] - cfg.xmin[d]) / (float(base[d]) * 16 * 1.0)
            ref = cfg.xmin[d] + (np.arange(bc * 16, bc * 16 + 16, dtype=np.float64) + 0.5) * dx
            line = {0: arr[b, 3, 5, :], 1: arr[b, 3, :, 5], 2: arr[b, :, 3, 5]}[d]
            assert np.array_equal(line, ref), (b, d)
