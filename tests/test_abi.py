"""The C ABI library builds, loads and exports every symbol that
include/dgsigma.h declares; host-only calls behave.  No device compute."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b((?:dg|sg)_\w+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_1907_06191_gb300 import _build
    _build.build()
    import paper_1907_06191_gb300 as dg
    return dg.lib()


def test_every_declared_symbol_is_exported(L):
    import paper_1907_06191_gb300 as dg
    names = _header_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(L, n), n
    assert sorted(dg.EXPORTS) == names


def test_host_only_calls(L):
    import paper_1907_06191_gb300 as dg
    assert L.dg_strerror(dg.DG_OK) == b"ok"
    assert L.dg_strerror(dg.DG_EUNSTABLE) == b"unstable time step"
    assert L.dg_strerror(99) == b"unknown status"
    cfg = dg.default_config()
    assert (cfg.p, cfg.precision, cfg.D, cfg.sigma0, cfg.cfl_safety) == (3, dg.DG_FP64, 2.0, 0.2, 0.9)
    assert L.dg_last_error(None) == b""
    L.dg_destroy(None)
    h = ctypes.c_void_p()
    bad = dg.default_config(p=9)
    assert L.dg_create(ctypes.byref(bad), ctypes.byref(h)) == dg.DG_EINVAL
    assert cfg.rounding == dg.DG_ROUND_STOCHASTIC
    bad = dg.default_config(rounding=5)
    assert L.dg_create(ctypes.byref(bad), ctypes.byref(h)) == dg.DG_EINVAL
    bad = dg.default_config(cfl_safety=1.5)
    assert L.dg_create(ctypes.byref(bad), ctypes.byref(h)) == dg.DG_EINVAL
    assert L.dg_create(None, ctypes.byref(h)) == dg.DG_EINVAL
    assert L.dg_step(None, 1, 1.0) == dg.DG_EINVAL
    # the switches refuse a null context before touching anything
    k = ctypes.c_int()
    for call, args in ((L.dg_set_launch, (0,)), (L.dg_set_contraction, (0,)),
                       (L.dg_set_triangle_fusion, (1,)), (L.dg_get_launch, (ctypes.byref(k),)),
                       (L.dg_get_contraction, (ctypes.byref(k),)),
                       (L.dg_get_triangle_fusion, (ctypes.byref(k),))):
        assert call(None, *args) == dg.DG_EINVAL
    # raster arguments are checked before any device call: a cell side that is
    # not a positive finite number is refused
    out = (ctypes.c_uint8 * 16)()
    one = (ctypes.c_double * 1)(1.0)
    for side in (0.0, -1.0, float("inf"), float("nan")):
        assert L.dg_rasterize_disks(one, one, one, 1, ctypes.c_double(side), 4, out) == dg.DG_EINVAL
    assert L.dg_rasterize_disks(one, one, one, 1, ctypes.c_double(2.0), 0, out) == dg.DG_EINVAL


def test_no_device_is_an_error_not_a_crash(L):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import paper_1907_06191_gb300 as dg
    h = ctypes.c_void_p()
    cfg = dg.default_config()
    assert L.dg_create(ctypes.byref(cfg), ctypes.byref(h)) == dg.DG_ECUDA
    assert not h.value
