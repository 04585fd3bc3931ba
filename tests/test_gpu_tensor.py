"""The p = 5 FP32 stage with its element contractions on the tensor cores
(tcgen05.mma, FP16 high/low split operands, FP32 accumulation; the remark of
Sec. 3.1: each element's update is a small dense local system).

Against the oracle on a walled mesh over 70 RK steps (a 64-step CUDA graph
plus 6 direct steps), node by node and on Sigma, for both FP32 roundings, the
penalty flux and the paper's wall mode; against the CUDA-core kernel and the
FP64 GPU path over long runs; mass conservation; the growing window; and the
bounded waits (test hook) ending in DG_ETIMEOUT with a usable context.  The
tolerance is the reduced-precision one (1e-4 relative); the measured errors
are printed."""
import numpy as np
import pytest

import dginputs
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402

TOL = 1e-4   # the reduced-precision path's bound on Sigma and on nodes (relative to max)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _mesh(seed=12):
    rng = np.random.default_rng(seed)
    act = (rng.random((37, 40)) > 0.3).astype(np.uint8)
    h, x0, y0 = 0.2, 0.5, -3.0
    src = []
    while len(src) < 3:
        ex, ey = int(rng.integers(8, 32)), int(rng.integers(8, 29))
        if act[ey, ex]:
            src.append((x0 + (ex + rng.uniform(0.1, 0.9)) * h, y0 + (ey + rng.uniform(0.1, 0.9)) * h))
    return act, h, x0, y0, np.array(src)


@pytest.mark.parametrize("rnd,eta,wall", [(dg.DG_ROUND_STOCHASTIC, 0.0, dg.DG_WALL_REMOVED),
                                          (dg.DG_ROUND_NEAREST, 0.0, dg.DG_WALL_REMOVED),
                                          (dg.DG_ROUND_STOCHASTIC, 1.0, dg.DG_WALL_REMOVED),
                                          (dg.DG_ROUND_STOCHASTIC, 0.0, dg.DG_WALL_PAPER)])
def test_tensor_core_steps_parity(rnd, eta, wall):
    act, h, x0, y0, src = _mesh()
    D, s0 = 2.0, 0.25
    mesh = O.Mesh(p=5, active=act, h=h, x0=x0, y0=y0, k0=D, eta=eta, wall_mode=wall)
    nsteps, dt = 70, 0.85 * O.rk3_real_limit() / O.power_rho(mesh)
    out = {}
    for mode in (0, 1):
        with dg.DGSolver(p=5, precision=dg.DG_FP32, D=D, sigma0=s0, device=0, rounding=rnd,
                         eta=eta, wall_mode=wall) as s:
            s.set_geometry_mask(act, h, x0, y0)
            s.set_contraction(mode)
            s.set_sources(src)
            s.step(nsteps, dt)
            assert s.get_contraction() == mode
            out[mode] = (s.get_nodes(), s.covariance())
    fields = [O.rk3(mesh, O.init_gaussian(mesh, x, y, s0), nsteps, dt) for x, y in src]
    mom0 = np.array([O.moments(mesh, O.init_gaussian(mesh, x, y, s0), x, y) for x, y in src])
    mom = np.array([O.moments(mesh, f, x, y) for f, (x, y) in zip(fields, src)])
    s_ref, _, m_ref = O.aggregate(mom, mom0)
    nodes, (s3, mu, mass) = out[1]
    node_err = max(_rel(nodes[k], fields[k]) for k in range(len(src)))
    sig_err = _rel(s3, s_ref)
    cc_err = max(_rel(out[0][0][k], fields[k]) for k in range(len(src)))
    print(f"tensor cores: node {node_err:.2e} (CUDA cores {cc_err:.2e}), Sigma {sig_err:.2e}, "
          f"mass {_rel(mass, m_ref):.2e}")
    assert node_err < TOL and sig_err < TOL and _rel(mass, m_ref) < TOL


def test_tensor_core_long_run_against_fp64_and_mass():
    """6000 steps of three densities on an all-active periodic window (the
    setting of the FP32 long-run test): Sigma against the FP64 GPU path, and
    the mass of a walled periodic cell over 3000 steps."""
    nel, h = 96, 0.15625
    act = np.ones((nel, nel), np.uint8)
    c = nel * h / 2
    src = np.array([[c + 0.11, c - 0.07], [c - 0.2, c + 0.13], [c + 0.05, c + 0.31]])
    kw = dict(D=2.0, sigma0=0.2, boundary=dg.DG_BC_PERIODIC, device=0)
    out = {}
    for name, prec, mode in (("f64", dg.DG_FP64, 0), ("cc", dg.DG_FP32, 0), ("tc", dg.DG_FP32, 1)):
        with dg.DGSolver(p=5, precision=prec, **kw) as s:
            s.set_geometry_mask(act, h)
            s.set_contraction(mode)
            s.set_sources(src)
            if name == "f64":
                dt, _ = s.query_dt()
            s.step(6000, dt)
            out[name] = s.covariance()[0]
    err = {k: _rel(out[k], out["f64"]) for k in ("cc", "tc")}
    print("p = 5, Sigma vs FP64 after 6000 steps:", err)
    assert err["tc"] < TOL
    d = dginputs.gamma_disks(5, 4.0, 2.0, 0.15, n=12, min_gap=0.05)
    src = dginputs.sample_sources(6, d, 4, 0.0, 4.0, margin=0.25)
    with dg.DGSolver(p=5, precision=dg.DG_FP32, D=1.0, sigma0=0.3,
                     boundary=dg.DG_BC_PERIODIC, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        s.set_contraction(1)
        s.set_sources(src)
        mass0 = s.covariance()[2]
        dt, _ = s.query_dt()
        s.step(3000, dt)
        mass = s.covariance()[2]
    drift = np.abs(mass / mass0 - 1).max()
    print(f"tensor cores: mass drift over 3000 steps {drift:.2e}")
    assert drift < TOL


def test_tensor_core_growing_window_and_tuning():
    d = dginputs.gamma_disks(3, 4.0, 2.0, 0.15, n=8, min_gap=0.05)
    src = dginputs.sample_sources(4, d, 3, 0.0, 4.0, margin=0.25)
    res = {}
    for mode in (0, 1, -1):
        with dg.DGSolver(p=5, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as s:
            s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 3)
            s.set_contraction(mode)
            s.set_growing_window(3.0)
            s.set_sources(src)
            dt, _ = s.query_dt()
            s.step(70, dt)
            res[mode] = (s.get_nodes(), s.get_contraction())
    assert res[1][1] == 1 and res[-1][1] in (0, 1)
    assert _rel(res[1][0], res[0][0]) < TOL
    # the tuned choice is one of the two, bit for bit
    assert np.array_equal(res[-1][0], res[res[-1][1]][0])


def test_tensor_core_wait_that_runs_out_reports_etimeout():
    d = dginputs.gamma_disks(3, 4.0, 2.0, 0.15, n=8, min_gap=0.05)
    src = dginputs.sample_sources(4, d, 3, 0.0, 4.0, margin=0.25)
    with dg.DGSolver(p=5, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        s.set_contraction(1)
        s.set_sources(src)
        dt, _ = s.query_dt()
        s.debug_copies(2)
        s.step(1, dt)
        assert s.get_contraction() == 1
        with pytest.raises(dg.DgError) as ei:
            s.covariance()
        assert ei.value.code == dg.DG_ETIMEOUT
        s.debug_copies(0)
        s.set_sources(src)
        s.step(10, dt)
        got = s.get_nodes()
    with dg.DGSolver(p=5, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as f:
        f.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        f.set_contraction(1)
        f.set_sources(src)
        f.step(10, dt)
        assert np.array_equal(f.get_nodes(), got)


def test_contraction_mode_errors_and_other_orders():
    with dg.DGSolver(p=3, precision=dg.DG_FP32, device=0) as s:
        for bad in (-2, 2):
            with pytest.raises(dg.DgError) as ei:
                s.set_contraction(bad)
            assert ei.value.code == dg.DG_EINVAL
        act = np.ones((20, 20), np.uint8)
        s.set_geometry_mask(act, 0.2)
        s.set_contraction(1)
        s.set_sources(np.array([[2.0, 2.0]]))
        dt, _ = s.query_dt()
        s.step(2, dt)
        assert s.get_contraction() == 0   # only p = 5 has the tensor-core kernel
