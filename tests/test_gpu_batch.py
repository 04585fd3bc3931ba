"""Batched geometries (several substrates advanced by one launch per stage).

Through the C ABI: a batch of uneven geometries (different cell sizes,
element sides and disk sets) must give, per geometry, the same node values as
a context holding that geometry alone (bit for bit: the per-element
arithmetic is identical), and must match the oracle run on each geometry
(FP64 1e-10 on nodes and Sigma).
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


def _geometries():
    # (seed, L, n_cell, tiles, n_disks): uneven sizes and element sides
    spec = [(1, 4.0, 16, 3, 4), (2, 6.0, 20, 1, 7), (3, 3.0, 16, 3, 2)]
    out = []
    for seed, L, nc, tiles, nd in spec:
        d = dginputs.gamma_disks(seed, L, 2.0, 0.3, n=nd, min_gap=0.05)
        h = L / nc
        lo, hi = (0.0, L) if tiles > 1 else (2.5 * h, L - 2.5 * h)
        src = dginputs.sample_sources(seed + 11, d, 3, lo, hi, margin=h)
        out.append((d, L, nc, tiles, src))
    return out


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batch_equals_single_contexts_and_oracle(prec):
    geos = _geometries()
    P = dg.DG_FP64 if prec == "f64" else dg.DG_FP32
    p, D, s0 = 2, 1.0, 0.3
    # a step that is stable on every geometry, from the oracle's own bound
    meshes, rho = [], 0.0
    for d, L, nc, tiles, _ in geos:
        act = O.window_mask(O.mask_disks(L, nc, d.cx, d.cy, d.r), tiles)
        m = O.Mesh(p=p, active=act, h=L / nc, x0=-(tiles // 2) * L, y0=-(tiles // 2) * L, k0=D)
        meshes.append(m)
        rho = max(rho, O.power_rho(m))
    nsteps, dt = 70, 0.8 * O.rk3_real_limit() / rho
    with dg.DGSolver(p=p, precision=P, D=D, sigma0=s0, device=0) as b:
        b.set_geometry_batch([(d.cx, d.cy, d.r) for d, *_ in geos],
                             [g[1] for g in geos], [g[2] for g in geos], [g[3] for g in geos])
        inf = b.info()
        assert inf.n_geometries == 3
        assert inf.n_elements_padded % 128 == 0  # each geometry padded to whole chunks
        b.set_sources(np.stack([g[4] for g in geos]))
        b.step(nsteps, dt)
        s3, mu, mass = b.covariance_batch()
        mom = b.moments().reshape(3, 3, 6)
        picks = [(g, s, ex, ey) for g, m in enumerate(meshes) for s in range(3)
                 for ex, ey in ((m.nx // 2, m.ny // 2), (1, 2), (m.nx - 2, m.ny - 3))]
        got = b.get_elements_batch(picks)
    tol = 1e-10 if prec == "f64" else 1e-5
    for g, ((d, L, nc, tiles, src), mesh) in enumerate(zip(geos, meshes)):
        with dg.DGSolver(p=p, precision=P, D=D, sigma0=s0, device=0) as one:
            one.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
            one.set_sources(src)
            one.step(nsteps, dt)
            single = one.get_nodes()
            s_one = one.covariance()[0]
        for q, (gg, s, ex, ey) in enumerate(picks):
            if gg == g:
                assert np.array_equal(got[q], single[s, ey, ex])
        assert np.abs(s3[g] - s_one).max() <= 1e-12 * np.abs(s_one).max()
        fields0 = [O.init_gaussian(mesh, x, y, s0) for x, y in src]
        fields = [O.rk3(mesh, f, nsteps, dt) for f in fields0]
        for s in range(3):
            assert np.abs(single[s] - fields[s]).max() <= tol * np.abs(fields[s]).max()
        mom0 = np.array([O.moments(mesh, f, x, y) for f, (x, y) in zip(fields0, src)])
        momr = np.array([O.moments(mesh, f, x, y) for f, (x, y) in zip(fields, src)])
        s_ref, mu_ref, m_ref = O.aggregate(momr, mom0)
        assert np.abs(s3[g] - s_ref).max() <= tol * np.abs(s_ref).max()
        assert np.abs(mass[g] - m_ref).max() <= tol * np.abs(m_ref).max()
        assert np.abs(mom[g] - momr).max() <= (tol if prec == "f64" else 1e-4) * np.abs(momr).max()


def test_batch_checkpoint_and_dt():
    geos = _geometries()
    with dg.DGSolver(p=3, precision=dg.DG_FP64, D=1.0, sigma0=0.3, device=0) as a:
        a.set_geometry_batch([(d.cx, d.cy, d.r) for d, *_ in geos],
                             [g[1] for g in geos], [g[2] for g in geos], [g[3] for g in geos])
        a.set_sources(np.stack([g[4] for g in geos]))
        dt, rho = a.query_dt()
        # the finest geometry (element side 0.1875) sets the bound
        for d, L, nc, tiles, src in geos:
            with dg.DGSolver(p=3, precision=dg.DG_FP64, D=1.0, sigma0=0.3, device=0) as one:
                one.set_geometry_disks(d.cx, d.cy, d.r, L, nc, tiles)
                one.set_sources(src)
                assert one.query_dt()[1] <= rho * 1.01
        a.step(10, dt)
        blob = a.get_state()
        a.step(10, dt)
        ref = a.covariance_batch()[0]
    with dg.DGSolver(p=3, precision=dg.DG_FP64, D=1.0, sigma0=0.3, device=0) as b:
        b.set_geometry_batch([(d.cx, d.cy, d.r) for d, *_ in geos],
                             [g[1] for g in geos], [g[2] for g in geos], [g[3] for g in geos])
        b.set_state(blob)
        b.step(10, dt)
        assert np.array_equal(b.covariance_batch()[0], ref)
