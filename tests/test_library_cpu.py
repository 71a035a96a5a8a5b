"""CPU checks of the C ABI library: it builds for sm_103a, loads, exports every symbol that
include/agile.h declares, and its host-side argument checks and allocator-failure handling
return status codes without touching a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "agile.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2607_19277_gb300 import agile, build
    if not os.path.exists(agile.LIB_PATH):
        build.build()
    return agile.load()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(agile_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert "agile_step" in syms and "agile_mesh_create" in syms
    for s in syms:
        assert hasattr(lib, s), s
    from paper_2607_19277_gb300 import agile
    assert sorted(agile.EXPORTS) == syms


def test_version(lib):
    assert b"sm_103a" in lib.agile_version()


@pytest.mark.parametrize("field,value", [("physics", 7), ("rk", 4), ("real_bytes", 2),
                                         ("gamma", 1.0), ("max_level", 0), ("limiter", 3),
                                         ("eos", 2)])
def test_invalid_config_rejected_on_host(lib, field, value):
    from paper_2607_19277_gb300 import agile
    cfg = agile.make_config()
    setattr(cfg, field, value)
    out = C.c_void_p()
    st = lib.agile_mesh_create(C.byref(cfg), None, None, C.byref(out))
    assert st == 1 and not out.value     # AGILE_EINVAL


def test_resistivity_only_for_mhd_and_non_negative(lib):
    from paper_2607_19277_gb300 import agile
    out = C.c_void_p()
    for kw in (dict(physics="hd", eta=0.1), dict(physics="mhd", eta=-1.0), dict(physics="mhd", eta=float("nan"))):
        cfg = agile.make_config(**kw)
        assert lib.agile_mesh_create(C.byref(cfg), None, None, C.byref(out)) == 1, kw
        assert not out.value
    cfg = agile.make_config(physics="mhd", eta=0.1)
    batch = C.c_void_p()
    assert lib.agile_batch_create(C.byref(cfg), 1, None, None, C.byref(batch)) == 1   # meshes only


def test_half_periodic_and_srhd_hll_rejected(lib):
    from paper_2607_19277_gb300 import agile
    out = C.c_void_p()
    cfg = agile.make_config(bc=("periodic", "outflow", "periodic", "periodic", "periodic", "periodic"))
    assert lib.agile_mesh_create(C.byref(cfg), None, None, C.byref(out)) == 1
    cfg = agile.make_config(physics="srhd", flux="hll")
    assert lib.agile_mesh_create(C.byref(cfg), None, None, C.byref(out)) == 1
    cfg = agile.make_config(physics="hd", eos="synge")    # the Synge EOS is srhd-only
    assert lib.agile_mesh_create(C.byref(cfg), None, None, C.byref(out)) == 1
    cfg = agile.make_config(physics="ffhd", flux="hll")    # ffhd: TVDLF only
    assert lib.agile_mesh_create(C.byref(cfg), None, None, C.byref(out)) == 1
    cfg = agile.make_config(physics="ffhd", flux="tvdlf", max_level=2)   # ffhd: uniform meshes
    assert lib.agile_mesh_create(C.byref(cfg), None, None, C.byref(out)) == 1


def test_allocator_failure_returns_enomem(lib):
    """A caller-supplied allocator that fails: creation reports AGILE_ENOMEM cleanly."""
    from paper_2607_19277_gb300 import agile
    calls = []

    def alloc(n, stream, ctx):
        calls.append(n)
        return None

    def free(p, stream, ctx):
        raise AssertionError("nothing was allocated")

    a = agile.agile_allocator(agile.ALLOC_FN(alloc), agile.FREE_FN(free), None)
    out = C.c_void_p()
    st = lib.agile_mesh_create(C.byref(agile.make_config()), C.byref(a), None, C.byref(out))
    assert st == 2 and not out.value     # AGILE_ENOMEM
    assert len(calls) >= 1


def test_binding_refuses_missing_library(tmp_path):
    from paper_2607_19277_gb300 import agile
    saved = agile._lib
    agile._lib = None
    try:
        with pytest.raises(OSError):
            agile.load(str(tmp_path / "missing.so"))
    finally:
        agile._lib = saved


@pytest.mark.parametrize("bad", [0.0, 5e-324, float("inf"), float("nan"), 2.0 ** 1022])
def test_rcp64_selftest_rejects_divisors_outside_its_range(lib, bad):
    """The quotient check validates its divisors on the host (zero, subnormal, infinite, NaN,
    or |s| >= 2^1022 are outside the documented range) before any device work."""
    import numpy as np
    from paper_2607_19277_gb300 import agile
    s = np.array([1.0, bad, 3.0])
    a = np.ones(3)
    with pytest.raises(agile.AgileError) as e:
        agile.check_rcp64(s, a)
    assert e.value.status == 1


def test_conduction_config_checked_on_host(lib):
    """ffhd with conduction: TVDLF only, uniform meshes, a finite kappa0 >= 0."""
    from paper_2607_19277_gb300 import agile
    out = C.c_void_p()
    for kw in (dict(flux="hll"), dict(max_level=2), dict(htc_kappa0=-1.0), dict(htc_kappa0=float("nan"))):
        args = dict(physics="ffhd_htc", flux="tvdlf", htc_kappa0=0.1)
        args.update(kw)
        cfg = agile.make_config(**args)
        assert lib.agile_mesh_create(C.byref(cfg), None, None, C.byref(out)) == 1, kw
