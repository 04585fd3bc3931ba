"""Chunks with more out-of-chunk face neighbours than a block has threads.

A stage kernel block owns one chunk of 128 consecutive elements and gives
each thread one entry of the chunk's halo list; entries beyond the first 128
are taken by a second loop.  The mesh here keeps only the rows on both sides
of every 16-row tile boundary, so every element of an interior chunk has its
vertical neighbour in another chunk: 130 halo entries per interior chunk (two
in the second loop).  Checked: the operator against the oracle for p = 1, 3,
5 in both precisions; SSP-RK3 steps against the oracle, with the p = 5
tensor-core contraction as well; every launch shape bit for bit.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402

H, X0, Y0, D, S0 = 0.25, -1.0, 0.5, 1.3, 0.3


def _band_mesh(nx=128, ny=64):
    act = np.zeros((ny, nx), np.uint8)
    for y in range(ny):
        if y % 16 in (0, 15):
            act[y] = 1
    return act


def _sources(act, m, seed=5):
    rng = np.random.default_rng(seed)
    ys, xs = np.nonzero(act)
    keep = (xs > 8) & (xs < act.shape[1] - 8) & (ys > 0) & (ys < act.shape[0] - 1)
    pick = rng.choice(np.flatnonzero(keep), size=m, replace=False)
    return np.stack([X0 + (xs[pick] + 0.5) * H, Y0 + (ys[pick] + 0.5) * H], axis=1)


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _solver(p, prec, **kw):
    return dg.DGSolver(p=p, precision=dg.DG_FP64 if prec == "f64" else dg.DG_FP32, D=D,
                       sigma0=S0, device=0, **kw)


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_operator_with_halo_beyond_one_entry_per_thread(p, prec):
    act = _band_mesh()
    mesh = O.Mesh(p=p, active=act, h=H, x0=X0, y0=Y0, k0=D)
    rng = np.random.default_rng(11 + p)
    m = 2
    u = rng.standard_normal((m,) + mesh.field_shape) * act[None, :, :, None, None]
    with _solver(p, prec) as s:
        s.set_geometry_mask(act, H, X0, Y0)
        assert s.info().halo_max > 128  # more halo entries than threads in a block
        s.set_sources(_sources(act, m))
        s.set_nodes(u)
        s.apply_operator()
        got = s.get_nodes()
    tol = 1e-12 if prec == "f64" else 2e-5
    for k in range(m):
        assert _rel(got[k], O.apply_L(mesh, u[k])) < tol


@pytest.mark.parametrize("p, contraction", [(3, 0), (5, 0), (5, 1)])
def test_rk3_steps_with_halo_beyond_one_entry_per_thread(p, contraction):
    act = _band_mesh()
    mesh = O.Mesh(p=p, active=act, h=H, x0=X0, y0=Y0, k0=D)
    src = _sources(act, 3)
    nsteps = 12
    with _solver(p, "f32") as s:
        s.set_geometry_mask(act, H, X0, Y0)
        s.set_contraction(contraction)
        s.set_sources(src)
        u0 = s.get_nodes()
        dt, _ = s.query_dt()
        s.step(nsteps, dt)
        got = s.get_nodes()
    # the suite's FP32 tolerances: CUDA cores 1e-5, the tensor-core split 1e-4
    tol = 1e-4 if contraction else 1e-5
    for k, (x, y) in enumerate(src):
        assert _rel(u0[k], O.init_gaussian(mesh, x, y, S0)) < 1e-7
        ref = O.rk3(mesh, u0[k], nsteps, dt)
        assert _rel(got[k], ref) < tol


def test_launch_shapes_agree_with_halo_beyond_one_entry_per_thread():
    act = _band_mesh()
    src = _sources(act, 4)
    out = {}
    for launch in (0, 2, -2):
        with _solver(3, "f32") as s:
            s.set_geometry_mask(act, H, X0, Y0)
            s.set_launch(launch)
            s.set_sources(src)
            dt, _ = s.query_dt()
            s.step(20, dt)
            out[launch] = (s.get_nodes(), s.get_launch())
    assert out[2][1] >= 1 and out[-2][1] == -2
    assert np.array_equal(out[0][0], out[2][0])
    assert np.array_equal(out[0][0], out[-2][0])
