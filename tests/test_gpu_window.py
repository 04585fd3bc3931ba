"""Growing window (dg_set_growing_window) through the C ABI.

The oracle's rk3_growing takes the same decisions (FP64 squared distance of
each element centre to the start-point box against r^2 (sigma0^2 + 2 D t) at
the end of each group of 64 steps) and holds the other elements, so the
CUDA path must match it node by node (FP64 1e-10, FP32 1e-5 of the field
maximum), hold those elements bit for bit, and reduce to the fixed window
when the radius covers the mesh.
"""
import numpy as np
import pytest

import dginputs
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402

PREC = {"f64": dg.DG_FP64, "f32": dg.DG_FP32}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1907_06191_gb300 import _build
    _build.build()
    O.build()


def _case(seed=3, L=4.0, nc=16, tiles=3, m=3):
    d = dginputs.gamma_disks(seed, L, 2.0, 0.15, n=10, min_gap=0.05)
    h = L / nc
    src = dginputs.sample_sources(seed + 1, d, m, 0.0, L, margin=h)
    act = O.mask_disks(L, nc, d.cx, d.cy, d.r)
    act = O.window_mask(act, tiles)
    return d, L, nc, tiles, src, act, h


def _box(src):
    return (src[:, 0].min(), src[:, 0].max(), src[:, 1].min(), src[:, 1].max())


@pytest.mark.parametrize("prec,p", [("f64", 2), ("f64", 3), ("f32", 3)])
def test_growing_window_matches_oracle(prec, p):
    d, L, nc, tiles, src, act, h = _case()
    D, s0, r = 1.0, 0.3, 3.0
    mesh = O.Mesh(p=p, active=act, h=h, x0=-(tiles // 2) * L, y0=-(tiles // 2) * L, k0=D)
    nsteps = 300
    dt = 0.8 * O.rk3_real_limit() / O.power_rho(mesh)
    with dg.DGSolver(p=p, precision=PREC[prec], D=D, sigma0=s0, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
        s.set_growing_window(r)
        s.set_sources(src)
        init = s.get_nodes()
        s.step(nsteps, dt)
        got = s.get_nodes()
    box = _box(src)
    d2 = O.window_d2(mesh, box)
    r2_end = r * r * (s0 * s0 + 2.0 * D * nsteps * dt)
    held = (act != 0) & (d2 > r2_end)
    assert held.sum() > 0.3 * act.sum()          # the window is still growing
    tol = 1e-10 if prec == "f64" else 1e-5
    for k, (x, y) in enumerate(src):
        ref = O.rk3_growing(mesh, O.init_gaussian(mesh, x, y, s0), nsteps, dt, box, r, s0)
        assert np.abs(got[k] - ref).max() <= tol * np.abs(ref).max()
        # held elements keep their start values bit for bit
        assert np.array_equal(got[k][held], init[k][held])


def test_large_radius_is_the_fixed_window_and_checkpoint():
    d, L, nc, tiles, src, act, h = _case()
    kw = dict(p=3, precision=dg.DG_FP64, D=1.0, sigma0=0.3, device=0)
    with dg.DGSolver(**kw) as a, dg.DGSolver(**kw) as b:
        for s in (a, b):
            s.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
            s.set_sources(src)
        dt, _ = a.query_dt()
        b.set_growing_window(1e3)
        a.step(150, dt)
        b.step(150, dt)
        assert np.array_equal(a.get_nodes(), b.get_nodes())
    # checkpoint in the middle of a growing-window run
    with dg.DGSolver(**kw) as a:
        a.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
        a.set_growing_window(3.0)
        a.set_sources(src)
        dt, _ = a.query_dt()
        a.step(100, dt)
        blob = a.get_state()
        a.step(100, dt)
        ref = a.get_nodes()
    with dg.DGSolver(**kw) as b:
        b.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
        b.set_growing_window(3.0)
        b.set_state(blob)
        b.step(100, dt)
        assert np.array_equal(b.get_nodes(), ref)


def test_window_then_fixed_then_window():
    """Switching the window off and on again: every switch resynchronises the
    stage arrays, so the result equals the oracle's schedule of the same
    calls."""
    d, L, nc, tiles, src, act, h = _case(m=2)
    D, s0 = 1.0, 0.3
    mesh = O.Mesh(p=2, active=act, h=h, x0=-(tiles // 2) * L, y0=-(tiles // 2) * L, k0=D)
    dt = 0.8 * O.rk3_real_limit() / O.power_rho(mesh)
    with dg.DGSolver(p=2, precision=dg.DG_FP64, D=D, sigma0=s0, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
        s.set_sources(src)
        s.set_growing_window(2.5)
        s.step(70, dt)
        s.set_growing_window(0.0)
        s.step(10, dt)
        s.set_growing_window(2.5)
        s.step(70, dt)
        got = s.get_nodes()
    box = _box(src)
    for k, (x, y) in enumerate(src):
        u = O.init_gaussian(mesh, x, y, s0)
        u = O.rk3_growing(mesh, u, 70, dt, box, 2.5, s0)
        u = O.rk3(mesh, u, 10, dt)
        u = O.rk3_growing(mesh, u, 70, dt, box, 2.5, s0, t0=70 * dt + 10 * dt)
        assert np.abs(got[k] - u).max() <= 1e-10 * np.abs(u).max()


def test_batched_geometries_use_their_own_boxes():
    geos = []
    for seed, L, nc in ((1, 4.0, 16), (2, 3.0, 12)):
        d = dginputs.gamma_disks(seed, L, 2.0, 0.15, n=6, min_gap=0.05)
        src = dginputs.sample_sources(seed + 5, d, 2, 0.0, L, margin=L / nc)
        geos.append((d, L, nc, 3, src))
    kw = dict(p=2, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0)
    with dg.DGSolver(**kw) as b:
        b.set_geometry_batch([(d.cx, d.cy, d.r) for d, *_ in geos], [g[1] for g in geos],
                             [g[2] for g in geos], [g[3] for g in geos])
        b.set_growing_window(3.0)
        b.set_sources(np.stack([g[4] for g in geos]))
        dt, _ = b.query_dt()
        b.step(200, dt)
        picks = [(g, s, ex, ey) for g in range(2) for s in range(2)
                 for ex, ey in ((20, 20), (24, 17), (5, 30))]
        got = b.get_elements_batch(picks)
    for g, (d, L, nc, tiles, src) in enumerate(geos):
        with dg.DGSolver(**kw) as one:
            one.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
            one.set_growing_window(3.0)
            one.set_sources(src)
            one.step(200, dt)
            single = one.get_nodes()
        for q, (gg, s, ex, ey) in enumerate(picks):
            if gg == g:
                assert np.array_equal(got[q], single[s, ey, ex])


@pytest.mark.parametrize("p,r,tol", [(2, 7.0, 1e-7), (3, 10.0, 1e-7)])
def test_propagate_sigma_close_to_fixed_window(p, r, tol):
    """Sigma of a growing-window solve against the fixed window.  The oracle
    gives, for these meshes (sigma0 = 1.2 h), 1.6e-8 at p = 2, r = 7 and
    8.5e-9 at p = 3, r = 10: odd p with the central fluxes has a heavier
    than Gaussian tail (4e-6 at p = 3, r = 7)."""
    d, L, nc, tiles, src, act, h = _case(m=4)
    kw = dict(p=p, precision=dg.DG_FP64, D=1.0, sigma0=0.3, device=0)
    out = []
    for rf in (0.0, r):
        with dg.DGSolver(**kw) as s:
            s.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
            s.set_growing_window(rf)
            s.set_sources(src)
            s.propagate_to(0.4)
            out.append(s.covariance()[0])
    assert np.abs(out[1] - out[0]).max() <= tol * np.abs(out[0]).max()


def test_bad_radius():
    with dg.DGSolver(p=2, device=0) as s:
        with pytest.raises(dg.DgError):
            s.set_growing_window(-1.0)
        with pytest.raises(dg.DgError):
            s.set_growing_window(float("nan"))
