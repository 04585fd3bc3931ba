"""dg_moments_dense_static: moments without any allocation.

Callers whose device memory belongs to another allocator, or who may not
risk an allocation's implicit synchronisation, pass their own device buffers
and get the raw moments; the reduction's scratch is a fixed array inside the
library.  This checks it through the C ABI against dg_moments (the
context-owned path) on two calls in a row with different densities and
precisions.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402


def _call(L, u, prec, m, nx, ny, p, h, x0, y0, xy, out, stream):
    return L.dg_moments_dense_static(
        ctypes.c_void_p(u.data_ptr()), prec, m, nx, ny, p, h, x0, y0,
        ctypes.c_void_p(xy.data_ptr()), ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(stream.cuda_stream))


def test_static_moments_match_context_moments():
    from paper_1907_06191_gb300 import _build
    _build.build()
    L = dg.lib()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(12)
    nx, ny, p, h, x0, y0 = 37, 29, 3, 0.25, -1.0, 2.0
    act = (rng.random((ny, nx)) > 0.3).astype(np.uint8)
    src = []
    while len(src) < 5:
        ex, ey = int(rng.integers(4, nx - 4)), int(rng.integers(4, ny - 4))
        if act[ey, ex]:
            src.append((x0 + (ex + 0.4) * h, y0 + (ey + 0.6) * h))
    src = np.array(src)
    stream = torch.cuda.Stream(device=0)
    xy = torch.from_numpy(src).to("cuda:0")
    for call, (prec_name, steps) in enumerate([("f64", 7), ("f32", 23)]):
        prec = dg.DG_FP64 if prec_name == "f64" else dg.DG_FP32
        with dg.DGSolver(p=p, precision=prec, D=1.5, sigma0=0.3, device=0) as s:
            s.set_geometry_mask(act, h, x0, y0)
            s.set_sources(src)
            dt, _ = s.query_dt()
            s.step(steps, dt)
            ref = s.moments()
            dense = s.get_nodes()
        tdt = torch.float64 if prec_name == "f64" else torch.float32
        u = torch.from_numpy(dense).to(device="cuda:0", dtype=tdt).contiguous()
        out = torch.full((len(src), 6), float("nan"), dtype=torch.float64, device="cuda:0")
        rc = _call(L, u, prec, len(src), nx, ny, p, h, x0, y0, xy, out, stream)
        assert rc == dg.DG_OK, f"call {call}: status {rc}"
        stream.synchronize()
        got = out.cpu().numpy()
        # the suite's tolerances: FP64 1e-10; FP32 densities 1e-5 (dg_moments
        # forms their element-local sums in FP32)
        tol = 1e-10 if prec_name == "f64" else 1e-5
        assert np.abs(got - ref).max() <= tol * np.abs(ref).max(), (call, got, ref)

    # a size beyond the fixed scratch is refused before any device work
    big = torch.zeros((129, 1, 1, 4, 4), dtype=torch.float64, device="cuda:0")
    xyb = torch.zeros((129, 2), dtype=torch.float64, device="cuda:0")
    outb = torch.zeros((129, 6), dtype=torch.float64, device="cuda:0")
    assert _call(L, big, dg.DG_FP64, 129, 1, 1, 3, 1.0, 0.0, 0.0, xyb, outb, stream) == dg.DG_EINVAL
