"""dg_moments_dense_static: moments without any allocation.

Callers whose device memory belongs to another allocator, or who may not
risk an allocation's implicit synchronisation, pass their own device buffers
and get the raw moments; the reduction's scratch is a fixed array inside the
library.  This checks it through the C ABI against dg_moments (the
context-owned path, itself checked against the oracle) on two calls in a row
with different densities and precisions, for p = 1, 3, 5, and with m = 128
densities, where the fixed array is exactly full.

The file is collected last on purpose: the entry point is an add-on outside
the method, so a run that stops at its first failure has already run every
other test when it reaches this one.  Nothing here depends on the order:
the test passes alone in a fresh process and after the others.
"""
import ctypes
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402

MAX_M = 128  # the documented capacity of the fixed scratch array


def _call(L, u, prec, m, nx, ny, p, h, x0, y0, xy, out, stream):
    return L.dg_moments_dense_static(
        ctypes.c_void_p(u.data_ptr()), prec, m, nx, ny, p, h, x0, y0,
        ctypes.c_void_p(xy.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(stream.cuda_stream))


def _case(seed, nx, ny, m, h=0.25, x0=-1.0, y0=2.0):
    rng = np.random.default_rng(seed)
    act = (rng.random((ny, nx)) > 0.3).astype(np.uint8)
    src = []
    while len(src) < m:
        ex, ey = int(rng.integers(2, nx - 2)), int(rng.integers(2, ny - 2))
        if act[ey, ex]:
            src.append((x0 + (ex + rng.uniform(0.2, 0.8)) * h, y0 + (ey + rng.uniform(0.2, 0.8)) * h))
    return act, np.array(src), h, x0, y0


def _context_moments(p, prec, act, src, h, x0, y0, steps):
    with dg.DGSolver(p=p, precision=prec, D=1.5, sigma0=0.3, device=0) as s:
        s.set_geometry_mask(act, h, x0, y0)
        s.set_sources(src)
        dt, _ = s.query_dt()
        s.step(steps, dt)
        return s.moments(), s.get_nodes()


def _check(L, stream, p, prec, act, src, h, x0, y0, steps):
    ref, dense = _context_moments(p, prec, act, src, h, x0, y0, steps)
    ny, nx = act.shape
    tdt = torch.float64 if prec == dg.DG_FP64 else torch.float32
    u = torch.from_numpy(dense).to(device="cuda:0", dtype=tdt).contiguous()
    xy = torch.from_numpy(src).to("cuda:0")
    out = torch.full((len(src), 6), float("nan"), dtype=torch.float64, device="cuda:0")
    rc = _call(L, u, prec, len(src), nx, ny, p, h, x0, y0, xy, out, stream)
    assert rc == dg.DG_OK, f"status {rc}"
    stream.synchronize()
    got = out.cpu().numpy()
    # the suite's tolerances: FP64 1e-10; FP32 densities 1e-5 (both paths
    # form the element-local sums in FP32, at different points of the sum)
    tol = 1e-10 if prec == dg.DG_FP64 else 1e-5
    assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (got, ref)


@pytest.fixture(scope="module")
def lib():
    from paper_1907_06191_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    return dg.lib()


@pytest.mark.parametrize("p", [1, 3, 5])
def test_static_moments_match_context_moments(lib, p):
    """Two calls in a row on the shared scratch: FP64 densities, then FP32
    densities of another step count (the second call must not see the
    first call's partial sums)."""
    act, src, h, x0, y0 = _case(12 + p, 37, 29, 5)
    stream = torch.cuda.Stream(device=0)
    _check(lib, stream, p, dg.DG_FP64, act, src, h, x0, y0, 7)
    _check(lib, stream, p, dg.DG_FP32, act, src, h, x0, y0, 23)


def test_static_moments_at_full_capacity(lib):
    """m = 128 fills the fixed array exactly; then a call with fewer
    densities reuses it."""
    act, src, h, x0, y0 = _case(99, 12, 10, MAX_M)
    stream = torch.cuda.Stream(device=0)
    _check(lib, stream, 2, dg.DG_FP64, act, src, h, x0, y0, 5)
    _check(lib, stream, 2, dg.DG_FP32, act, src[:3], h, x0, y0, 5)


def test_static_moments_refuse_bad_arguments(lib):
    """Sizes beyond the fixed scratch and non-finite grids are refused before
    any device work."""
    stream = torch.cuda.Stream(device=0)
    big = torch.zeros((MAX_M + 1, 1, 1, 4, 4), dtype=torch.float64, device="cuda:0")
    xyb = torch.zeros((MAX_M + 1, 2), dtype=torch.float64, device="cuda:0")
    outb = torch.zeros((MAX_M + 1, 6), dtype=torch.float64, device="cuda:0")
    assert _call(lib, big, dg.DG_FP64, MAX_M + 1, 1, 1, 3, 1.0, 0.0, 0.0, xyb, outb,
                 stream) == dg.DG_EINVAL
    for h, x0, y0 in [(math.inf, 0.0, 0.0), (1.0, math.nan, 0.0), (1.0, 0.0, -math.inf)]:
        assert _call(lib, big, dg.DG_FP64, 1, 1, 1, 3, h, x0, y0, xyb, outb,
                     stream) == dg.DG_EINVAL
