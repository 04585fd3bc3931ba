"""The stage kernel's shared-memory copies: one tensor copy (TMA) per chunk
with a hardware swizzle, or per-thread cp.async copies.  Both fill the same
layout, so the results must agree bit for bit; the tensor path must really
run where the element rows are whole 16-byte slots; and a barrier that never
completes (test hook) must end in DG_ETIMEOUT with a usable context.  The
time-out is made on the host side of the test: the barrier waits for bytes
that no copy delivers, and the kernel's bounded wait gives up."""
import numpy as np
import pytest

import dginputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402

PREC = {"f64": dg.DG_FP64, "f32": dg.DG_FP32}


def _case():
    d = dginputs.gamma_disks(3, 4.0, 2.0, 0.15, n=8, min_gap=0.05)
    src = dginputs.sample_sources(4, d, 3, 0.0, 4.0, margin=0.25)
    return d, src


def _run(p, prec, mode, nsteps=70, grow=0.0):
    d, src = _case()
    with dg.DGSolver(p=p, precision=PREC[prec], D=1.0, sigma0=0.3, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 3)
        s.set_growing_window(grow)
        s.set_sources(src)
        s.debug_copies(mode)
        dt, _ = s.query_dt()
        s.step(nsteps, dt)
        nodes = s.get_nodes()
        sig = s.covariance()[0]
        n = s.debug_copies(0)
    return nodes, sig, n


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_tensor_copies_equal_cp_async(p, prec):
    a, sa, na = _run(p, prec, 0)
    b, sb, nb = _run(p, prec, 1)
    assert na > 0 and nb == 0
    assert np.array_equal(a, b) and np.array_equal(sa, sb)


def test_tensor_copies_with_the_growing_window():
    a, _, na = _run(3, "f32", 0, grow=3.0)
    b, _, nb = _run(3, "f32", 1, grow=3.0)
    assert na > 0 and nb == 0
    assert np.array_equal(a, b)


@pytest.mark.parametrize("p", [2, 4])
def test_partial_slot_rows_use_cp_async(p):
    _, _, n = _run(p, "f32", 0, nsteps=3)
    assert n == 0


def test_wait_that_runs_out_reports_etimeout():
    d, src = _case()
    with dg.DGSolver(p=3, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        s.set_sources(src)
        dt, _ = s.query_dt()
        s.debug_copies(2)
        s.step(1, dt)
        with pytest.raises(dg.DgError) as ei:
            s.covariance()
        assert ei.value.code == dg.DG_ETIMEOUT
        # the context is usable again: new start densities and a normal step
        s.debug_copies(0)
        s.set_sources(src)
        s.step(10, dt)
        got = s.get_nodes()
        sig = s.covariance()[0]
    with dg.DGSolver(p=3, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as f:
        f.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        f.set_sources(src)
        f.step(10, dt)
        assert np.array_equal(f.get_nodes(), got)
        assert np.array_equal(f.covariance()[0], sig)


def test_bad_copy_mode():
    with dg.DGSolver(p=3, device=0) as s:
        with pytest.raises(dg.DgError):
            s.debug_copies(4)
