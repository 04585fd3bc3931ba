"""Launch shapes of the FP32 stage kernel (one block per chunk, or a
persistent launch whose blocks walk the (density, chunk) work items with the
next item's chunks copied in behind the current one).  Every shape must give
the same bits: the per-element arithmetic and its rounding keys do not depend
on which block runs an element.  Checked on a walled periodic-cell window
with the penalty on and off, both FP32 roundings, the growing window (a
chunk list and held elements) and a batch of geometries; the tuned shape is
one of the candidates; a bounded copy wait of the persistent kernel that
runs out (test hook) ends in DG_ETIMEOUT with a usable context."""
import numpy as np
import pytest

import dginputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402


def _case(seed=3):
    d = dginputs.gamma_disks(seed, 4.0, 2.0, 0.15, n=8, min_gap=0.05)
    src = dginputs.sample_sources(seed + 1, d, 5, 0.0, 4.0, margin=0.25)
    return d, src


def _run(p, launch, rnd=dg.DG_ROUND_STOCHASTIC, eta=0.0, grow=0.0, nsteps=70):
    d, src = _case()
    with dg.DGSolver(p=p, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0, rounding=rnd,
                     eta=eta) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 3)
        s.set_launch(launch)
        s.set_growing_window(grow)
        s.set_sources(src)
        dt, _ = s.query_dt()
        s.step(nsteps, dt)   # one 64-step graph + 6 direct steps
        return s.get_nodes(), s.covariance()[0], s.get_launch()


@pytest.mark.parametrize("p", [1, 3])
@pytest.mark.parametrize("rnd", [dg.DG_ROUND_STOCHASTIC, dg.DG_ROUND_NEAREST])
@pytest.mark.parametrize("eta", [0.0, 1.0])
def test_persistent_launch_gives_the_same_bits(p, rnd, eta):
    ref, sref, k0 = _run(p, 0, rnd, eta)
    assert k0 == 0
    for k in (1, 2, 3):
        got, sig, used = _run(p, k, rnd, eta)
        assert 1 <= used <= k
        assert np.array_equal(got, ref) and np.array_equal(sig, sref), k


@pytest.mark.parametrize("p", [1, 3])
def test_persistent_launch_with_the_growing_window(p):
    ref, _, _ = _run(p, 0, grow=3.0)
    got, _, used = _run(p, 2, grow=3.0)
    assert used >= 1
    assert np.array_equal(got, ref)


def test_tuned_launch_is_a_candidate_and_gives_the_same_bits():
    ref, sref, _ = _run(3, 0)
    got, sig, used = _run(3, -1)
    assert used >= 0
    assert np.array_equal(got, ref) and np.array_equal(sig, sref)


def test_persistent_launch_over_a_batch_of_geometries():
    ws = [dginputs.gamma_disks(s, 4.0, 2.0, 0.15, n=6 + s, min_gap=0.05) for s in range(3)]
    src = np.stack([dginputs.sample_sources(10 + s, d, 4, 0.0, 4.0, margin=0.25)
                    for s, d in enumerate(ws)])
    out = []
    for k in (0, 2):
        with dg.DGSolver(p=3, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as s:
            s.set_geometry_batch([(d.cx, d.cy, d.r) for d in ws], [4.0, 4.0, 4.0], [16, 20, 12],
                                 [3, 3, 3])
            s.set_launch(k)
            s.set_sources(src)
            dt, _ = s.query_dt()
            s.step(40, dt)
            out.append((s.covariance_batch()[0], s.get_launch()))
    assert out[1][1] >= 1
    assert np.array_equal(out[0][0], out[1][0])


def test_fp64_keeps_one_block_per_chunk():
    d, src = _case()
    with dg.DGSolver(p=3, precision=dg.DG_FP64, D=1.0, sigma0=0.3, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        s.set_launch(3)
        s.set_sources(src)
        dt, _ = s.query_dt()
        s.step(2, dt)
        assert s.get_launch() == 0


def test_persistent_wait_that_runs_out_reports_etimeout():
    d, src = _case()
    with dg.DGSolver(p=3, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        s.set_launch(2)
        s.set_sources(src)
        dt, _ = s.query_dt()
        s.debug_copies(2)
        s.step(1, dt)
        assert s.get_launch() >= 1
        with pytest.raises(dg.DgError) as ei:
            s.covariance()
        assert ei.value.code == dg.DG_ETIMEOUT
        s.debug_copies(0)
        s.set_sources(src)
        s.step(10, dt)
        got = s.get_nodes()
    with dg.DGSolver(p=3, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as f:
        f.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        f.set_launch(0)
        f.set_sources(src)
        f.step(10, dt)
        assert np.array_equal(f.get_nodes(), got)


def test_bad_launch_shape():
    with dg.DGSolver(p=3, device=0) as s:
        for bad in (-3, 65):
            with pytest.raises(dg.DgError) as ei:
                s.set_launch(bad)
            assert ei.value.code == dg.DG_EINVAL



STEP = -2  # DG_LAUNCH_STEP: the three stages of a step in one cooperative launch


@pytest.mark.parametrize("p", [1, 3, 5])
@pytest.mark.parametrize("rnd,eta", [(dg.DG_ROUND_STOCHASTIC, 0.0), (dg.DG_ROUND_NEAREST, 1.0)])
def test_one_launch_per_step_gives_the_same_bits(p, rnd, eta):
    ref, sref, _ = _run(p, 0, rnd, eta)
    got, sig, used = _run(p, STEP, rnd, eta)
    assert used == STEP
    assert np.array_equal(got, ref) and np.array_equal(sig, sref)


def test_one_launch_per_step_with_the_growing_window_and_a_batch():
    ref, _, _ = _run(3, 0, grow=3.0)
    got, _, used = _run(3, STEP, grow=3.0)
    assert used == STEP and np.array_equal(got, ref)
    ws = [dginputs.gamma_disks(s, 4.0, 2.0, 0.15, n=6 + s, min_gap=0.05) for s in range(3)]
    src = np.stack([dginputs.sample_sources(10 + s, d, 4, 0.0, 4.0, margin=0.25)
                    for s, d in enumerate(ws)])
    out = []
    for k in (0, STEP):
        with dg.DGSolver(p=3, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as s:
            s.set_geometry_batch([(d.cx, d.cy, d.r) for d in ws], [4.0, 4.0, 4.0], [16, 20, 12],
                                 [3, 3, 3])
            s.set_launch(k)
            s.set_sources(src)
            dt, _ = s.query_dt()
            s.step(40, dt)
            out.append(s.covariance_batch()[0])
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("mode", [2, 3])
def test_grid_barrier_or_copy_wait_that_runs_out_reports_etimeout(mode):
    """mode 3: every grid barrier waits for one block more than the launch
    has (a count nothing reaches); mode 2: the chunk copies' barriers wait
    for bytes no copy delivers.  Both bounded waits end in DG_ETIMEOUT and
    the context then reproduces a fresh run bit for bit."""
    d, src = _case()
    with dg.DGSolver(p=3, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as s:
        s.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        s.set_launch(STEP)
        s.set_sources(src)
        dt, _ = s.query_dt()
        s.debug_copies(mode)
        s.step(2, dt)
        assert s.get_launch() == STEP
        with pytest.raises(dg.DgError) as ei:
            s.covariance()
        assert ei.value.code == dg.DG_ETIMEOUT
        s.debug_copies(0)
        s.set_sources(src)
        s.step(10, dt)
        got = s.get_nodes()
    with dg.DGSolver(p=3, precision=dg.DG_FP32, D=1.0, sigma0=0.3, device=0) as f:
        f.set_geometry_disks(d.cx, d.cy, d.r, 4.0, 16, 1)
        f.set_launch(0)
        f.set_sources(src)
        f.step(10, dt)
        assert np.array_equal(f.get_nodes(), got)
