"""Failure paths through the C ABI, made on the host: an injected allocation
failure (dg_debug_fail_alloc) at every allocation of a whole solve must come
back as DG_ENOMEM, leave the context usable or destroyable, and leave no
trace in a later solve.  No GPU fault is involved."""
import numpy as np
import pytest

import dginputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402


@pytest.fixture(autouse=True)
def _disarm():
    dg.lib().dg_debug_fail_alloc(-1)
    yield
    dg.lib().dg_debug_fail_alloc(-1)


def _case():
    d = dginputs.gamma_disks(3, 4.0, 2.0, 0.15, n=8, min_gap=0.05)
    src = dginputs.sample_sources(4, d, 3, 0.0, 4.0, margin=0.25)
    return d, src


def _solve(d, src, grow=0.0):
    with dg.DGSolver(p=2, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 3)
        s.set_growing_window(grow)
        s.set_sources(src)
        dt, _ = s.query_dt()
        s.step(70, dt)
        return s.covariance()[0], s.get_nodes()


def test_every_allocation_failure_is_reported_and_harmless():
    d, src = _case()
    ref_sigma, ref_nodes = _solve(d, src, grow=3.0)
    failures = 0
    for k in range(200):
        dg.lib().dg_debug_fail_alloc(k)
        try:
            sigma, nodes = _solve(d, src, grow=3.0)
        except dg.DgError as e:
            assert e.code == dg.DG_ENOMEM, str(e)
            failures += 1
            continue
        finally:
            dg.lib().dg_debug_fail_alloc(-1)
        # k is past the last allocation: the solve is the reference, bit for bit
        assert np.array_equal(sigma, ref_sigma) and np.array_equal(nodes, ref_nodes)
        break
    else:
        pytest.fail("the solve never completed")
    assert failures >= 10          # geometry, sources, power iteration, window
    # and nothing leaked into a fresh solve
    sigma, nodes = _solve(d, src, grow=3.0)
    assert np.array_equal(nodes, ref_nodes)


def test_context_survives_a_failed_set_sources():
    d, src = _case()
    with dg.DGSolver(p=2, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 3)
        dt, _ = s.query_dt()
        dg.lib().dg_debug_fail_alloc(2)
        with pytest.raises(dg.DgError) as ei:
            s.set_sources(src)
        assert ei.value.code == dg.DG_ENOMEM
        dg.lib().dg_debug_fail_alloc(-1)
        with pytest.raises(dg.DgError) as ei:
            s.step(1, dt)                      # no sources after the failure
        assert ei.value.code == dg.DG_ESTATE
        s.set_sources(src)
        s.step(70, dt)
        nodes = s.get_nodes()
    assert np.array_equal(nodes, _solve(d, src)[1])


def test_bad_hook_argument():
    assert dg.lib().dg_debug_fail_alloc(-2) == dg.DG_EINVAL
