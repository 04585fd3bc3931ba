"""The paper's pixel triangles (DG_ELEMENT_TRIANGLE, Sec. 3.3) through the C
ABI against oracle/triangles.py: the operator alone, start densities, SSP-RK3
steps node by node, Sigma and mass (FP64 1e-10 relative to the field
maximum, 1e-12 for one operator application; FP32 1e-5, 2e-5 for the
operator), free diffusion 2Tk on the GPU, and the library's own tables."""
import numpy as np
import pytest

import dginputs
import oracle as O
from oracle import triangles as T

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


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _solver(p, prec, **kw):
    return dg.DGSolver(p=p, precision=PREC[prec], element=dg.DG_ELEMENT_TRIANGLE, device=0, **kw)


def _mesh(seed, nx, ny, frac=0.2):
    rng = np.random.default_rng(seed)
    act = (rng.random((ny, nx)) > frac).astype(np.uint8)
    return act, rng


def _sources(act, rng, m, h, x0, y0):
    ny, nx = act.shape
    out = []
    while len(out) < m:
        ex, ey = int(rng.integers(0, nx)), int(rng.integers(0, ny))
        if act[ey, ex]:
            out.append((x0 + (ex + rng.uniform(0.1, 0.9)) * h, y0 + (ey + rng.uniform(0.1, 0.9)) * h))
    return np.array(out)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("mode,per", [(0, False), (1, False), (0, True)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_operator_parity(p, mode, per, prec):
    act, rng = _mesh(7 + p, 13, 9)
    h, x0, y0, k0 = 0.3, -1.0, 0.5, 1.7
    mesh = T.TriMesh(p=p, active=act, h=h, x0=x0, y0=y0, k0=k0, wall_mode=mode, periodic=per)
    m = 2
    u = rng.standard_normal((m,) + mesh.shape) * act[None, :, :, None, None]
    with _solver(p, prec, D=k0, wall_mode=mode,
                 boundary=dg.DG_BC_PERIODIC if per else dg.DG_BC_ABSORBING) as s:
        s.set_geometry_mask(act, h, x0, y0)
        s.set_sources(_sources(act, rng, m, h, x0, y0))
        s.set_nodes(u)
        s.apply_operator()
        got = s.get_nodes()
    for k in range(m):
        ref = T.apply_L(mesh, u[k])
        assert _rel(got[k], ref) < (1e-12 if prec == "f64" else 2e-5)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_rk3_steps_and_sigma_parity(p, prec):
    act, rng = _mesh(20 + p, 23, 17)
    h, k0, s0 = 0.25, 1.0, 0.4
    mesh = T.TriMesh(p=p, active=act, h=h, k0=k0)
    src = _sources(act, rng, 3, h, 0.0, 0.0)
    dt = 0.8 * O.rk3_real_limit() / T.power_rho(mesh, iters=200)
    nsteps = 70                       # one 64-step graph and 6 direct steps
    with _solver(p, prec, D=k0, sigma0=s0) as s:
        s.set_geometry_mask(act, h)
        s.set_sources(src)
        init = s.get_nodes()
        s.step(nsteps, dt)
        got = s.get_nodes()
        sig, mu, mass = s.covariance()
        mom = s.moments()
    tol = 1e-10 if prec == "f64" else 1e-5
    f0 = [T.init_gaussian(mesh, x, y, s0) for x, y in src]
    fields = [T.rk3(mesh, f, nsteps, dt) for f in f0]
    for k in range(3):
        assert _rel(init[k], f0[k]) < (1e-14 if prec == "f64" else 1e-7)
        assert _rel(got[k], fields[k]) < tol
    m0 = np.array([T.moments(mesh, f, x, y) for f, (x, y) in zip(f0, src)])
    m1 = np.array([T.moments(mesh, f, x, y) for f, (x, y) in zip(fields, src)])
    s_ref, mu_ref, mass_ref = O.aggregate(m1, m0)
    assert _rel(sig, s_ref) < tol
    assert _rel(mass, mass_ref) < tol
    assert _rel(mom, m1) < (tol if prec == "f64" else 1e-4)


def test_spectral_radius_and_dt():
    """The library's power iteration (200 steps) against the exact spectral
    radius of the oracle's dense operator: from below, within 1% (the 0.9
    CFL safety factor covers the gap)."""
    act, rng = _mesh(3, 9, 8)
    mesh = T.TriMesh(p=2, active=act, h=0.3, k0=2.0)
    with _solver(2, "f64", D=2.0, sigma0=0.3) as s:
        s.set_geometry_mask(act, 0.3)
        s.set_sources(_sources(act, rng, 1, 0.3, 0.0, 0.0))
        dt, rho = s.query_dt()
    exact = np.abs(np.linalg.eigvals(T.dense_operator(mesh))).max()
    assert 0.99 * exact < rho <= exact * (1 + 1e-9)
    assert abs(dt - 0.9 * O.rk3_real_limit() / rho) < 1e-15


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_free_diffusion_on_triangles(prec):
    """Sigma = 2 D t for free diffusion (x^2 in P_2, L symmetric).  The
    oracle gives 8.1e-9 for this window (the heavier than Gaussian tail of
    the central fluxes reaching the edge)."""
    nel, h, D, s0 = 64, 0.5, 1.0, 1.0
    act = np.ones((nel, nel), np.uint8)
    c = nel * h / 2
    with _solver(2, prec, D=D, sigma0=s0) as s:
        s.set_geometry_mask(act, h)
        s.set_sources(np.array([[c + 0.13, c - 0.21], [c - 0.3, c + 0.05]]))
        s.propagate_to(1.0)
        sig = s.covariance()[0]
    tol = 3e-8 if prec == "f64" else 2e-6
    assert abs(sig[0] / 2.0 - 1) < tol and abs(sig[2] / 2.0 - 1) < tol and abs(sig[1]) < tol


def test_disk_window_and_batch():
    """A disk substrate tiled into a window, and two geometries in one batch:
    each geometry's nodes equal those of a context holding it alone."""
    geos = []
    for seed, L, nc in ((1, 4.0, 16), (2, 3.0, 12)):
        d = dginputs.gamma_disks(seed, L, 2.0, 0.15, n=6, min_gap=0.05)
        src = dginputs.sample_sources(seed + 5, d, 2, 0.0, L, margin=L / nc)
        geos.append((d, L, nc, 3, src))
    kw = dict(D=1.0, sigma0=0.3)
    with _solver(2, "f32", **kw) as b:
        b.set_geometry_batch([(d.cx, d.cy, d.r) for d, *_ in geos], [g[1] for g in geos],
                             [g[2] for g in geos], [g[3] for g in geos])
        b.set_sources(np.stack([g[4] for g in geos]))
        dt, _ = b.query_dt()
        b.step(80, dt)
        picks = [(g, s, ex, ey) for g in range(2) for s in range(2)
                 for ex, ey in ((20, 20), (24, 17), (5, 30))]
        got = b.get_elements_batch(picks)
    for g, (d, L, nc, tiles, src) in enumerate(geos):
        with _solver(2, "f32", **kw) as one:
            one.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
            one.set_sources(src)
            one.step(80, dt)
            single = one.get_nodes()
        for q, (gg, s, ex, ey) in enumerate(picks):
            if gg == g:
                assert np.array_equal(got[q], single[s, ey, ex])


def test_triangle_arguments():
    with pytest.raises(dg.DgError):
        _solver(4, "f64")
    with pytest.raises(dg.DgError):
        _solver(2, "f64", eta=1.0)
    act = np.ones((6, 6), np.uint8)
    with _solver(2, "f64", D=1.0, sigma0=0.3) as s:
        s.set_geometry_mask(act, 0.5)
        s.set_sources(np.array([[1.5, 1.5]]))
        with pytest.raises(dg.DgError):
            s.ls_residual()


def test_growing_window_on_triangles():
    """The growing window works on the triangle path too: a radius that
    covers the window is the fixed window bit for bit, and with a small
    radius the held pixels keep their start values bit for bit."""
    d = dginputs.gamma_disks(3, 4.0, 2.0, 0.15, n=8, min_gap=0.05)
    src = dginputs.sample_sources(4, d, 2, 0.0, 4.0, margin=0.25)
    kw = dict(D=1.0, sigma0=0.3)
    out = []
    for r in (0.0, 1e3, 2.0):
        with _solver(2, "f64", **kw) as s:
            s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 3)
            s.set_growing_window(r)
            s.set_sources(src)
            init = s.get_nodes()
            dt, _ = s.query_dt()
            s.step(90, dt)
            out.append((init, s.get_nodes(), dt))
    assert np.array_equal(out[0][1], out[1][1])
    init, grown, dt = out[2]
    box = (src[:, 0].min(), src[:, 0].max(), src[:, 1].min(), src[:, 1].max())
    L, nc, tiles = 4.0, 16, 3
    mesh = O.Mesh(p=1, active=np.ones((nc * tiles, nc * tiles), np.uint8), h=L / nc,
                  x0=-(tiles // 2) * L, y0=-(tiles // 2) * L)
    d2 = O.window_d2(mesh, box)
    held = d2 > 4.0 * (0.09 + 2.0 * 90 * dt)
    assert held.sum() > 100
    assert np.array_equal(grown[:, held], init[:, held])
    assert not np.array_equal(grown, out[0][1])
