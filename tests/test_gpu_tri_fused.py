"""The pixel-triangle stage as one launch (q kept in shared memory, the q of
each neighbouring triangle across a chunk boundary computed again in the
block) against the two-launch stage (q written to device memory and read
back): the same bits on random meshes with walls of both kinds, periodic
and absorbing boundaries, both FP32 roundings, chunks with more halo
entries than a block has threads, the growing window and the operator
alone; the operator on the many-halo mesh against the oracle too."""
import numpy as np
import pytest

from oracle import triangles as T

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402


def _solver(p, prec=dg.DG_FP32, **kw):
    return dg.DGSolver(p=p, precision=prec, element=dg.DG_ELEMENT_TRIANGLE, device=0, **kw)


def _random_mesh(seed, nx, ny, frac=0.2):
    rng = np.random.default_rng(seed)
    return (rng.random((ny, nx)) > frac).astype(np.uint8), rng


def _band_mesh(nx=128, ny=64):
    """Rows on both sides of every 16-row tile boundary: 130 halo entries per
    interior chunk of 128 pixels."""
    act = np.zeros((ny, nx), np.uint8)
    for y in range(ny):
        if y % 16 in (0, 15):
            act[y] = 1
    return act


def _sources(act, rng, m, h):
    ys, xs = np.nonzero(act)
    pick = rng.choice(len(xs), size=m, replace=False)
    return np.stack([(xs[pick] + 0.5) * h, (ys[pick] + 0.5) * h], axis=1)


def _steps(p, act, src, fused, nsteps=70, grow=0.0, **kw):
    with _solver(p, D=1.0, sigma0=0.3, **kw) as s:
        s.set_geometry_mask(act, 0.25)
        s.set_triangle_fusion(fused)
        s.set_growing_window(grow)
        s.set_sources(src)
        dt, _ = s.query_dt()
        s.step(nsteps, dt)   # one 64-step graph and direct steps
        return s.get_nodes(), s.covariance()[0], s.get_triangle_fusion()


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("rnd", [dg.DG_ROUND_STOCHASTIC, dg.DG_ROUND_NEAREST])
@pytest.mark.parametrize("mode,per", [(0, False), (1, False), (0, True)])
def test_one_launch_gives_the_bits_of_two(p, rnd, mode, per):
    act, rng = _random_mesh(31 + p, 40, 33)
    src = _sources(act, rng, 3, 0.25)
    kw = dict(rounding=rnd, wall_mode=mode,
              boundary=dg.DG_BC_PERIODIC if per else dg.DG_BC_ABSORBING)
    ref, sref, f0 = _steps(p, act, src, 0, **kw)
    got, sig, f1 = _steps(p, act, src, 1, **kw)
    assert (f0, f1) == (0, 1)
    assert np.array_equal(got, ref) and np.array_equal(sig, sref)


@pytest.mark.parametrize("p", [2, 3])
def test_one_launch_with_halo_beyond_one_entry_per_thread(p):
    act = _band_mesh()
    rng = np.random.default_rng(3)
    src = _sources(act, rng, 3, 0.25)
    ref, _, _ = _steps(p, act, src, 0, nsteps=20)
    got, _, _ = _steps(p, act, src, 1, nsteps=20)
    assert np.array_equal(got, ref)
    # the operator alone against the oracle on the same mesh
    mesh = T.TriMesh(p=p, active=act, h=0.25, k0=1.3)
    u = rng.standard_normal((2,) + mesh.shape) * act[None, :, :, None, None]
    with _solver(p, D=1.3) as s:
        s.set_geometry_mask(act, 0.25)
        assert s.info().halo_max > 128
        s.set_sources(src[:2])
        s.set_nodes(u)
        s.apply_operator()
        got = s.get_nodes()
    for k in range(2):
        ref = T.apply_L(mesh, u[k])
        assert np.abs(got[k] - ref).max() < 2e-5 * np.abs(ref).max()


def test_one_launch_with_the_growing_window():
    act, rng = _random_mesh(5, 48, 40, frac=0.1)
    src = _sources(act, rng, 2, 0.25)
    ref, _, _ = _steps(3, act, src, 0, grow=2.0)
    got, _, _ = _steps(3, act, src, 1, grow=2.0)
    assert np.array_equal(got, ref)


def test_operator_one_launch_equals_two():
    act, rng = _random_mesh(8, 21, 19)
    u = None
    out = []
    for fused in (0, 1):
        with _solver(3, D=1.7) as s:
            s.set_geometry_mask(act, 0.3)
            s.set_triangle_fusion(fused)
            s.set_sources(_sources(act, np.random.default_rng(1), 2, 0.3))
            if u is None:
                shape = (2,) + act.shape + tuple(s.node_shape())
                u = np.random.default_rng(2).standard_normal(shape) * act[None, :, :, None, None]
            s.set_nodes(u)
            s.apply_operator()
            out.append(s.get_nodes())
    assert np.array_equal(out[0], out[1])


def test_fusion_switch():
    act = np.ones((8, 8), np.uint8)
    for p, prec, want in ((1, dg.DG_FP32, 0), (2, dg.DG_FP32, 1), (3, dg.DG_FP32, 1),
                          (3, dg.DG_FP64, 0)):
        with _solver(p, prec, D=1.0, sigma0=0.3) as s:
            s.set_geometry_mask(act, 0.5)
            assert s.get_triangle_fusion() == want
            s.set_triangle_fusion(0)
            assert s.get_triangle_fusion() == 0
            with pytest.raises(dg.DgError):
                s.set_triangle_fusion(2)
    with dg.DGSolver(p=3, precision=dg.DG_FP32, device=0) as s:  # square elements
        assert s.get_triangle_fusion() == 0
