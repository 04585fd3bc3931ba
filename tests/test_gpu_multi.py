"""The sharded Sigma on the device (Sec. 4.1: start points are independent).

Start points split over several contexts (as over ranks), their raw moments
concatenated and handed to ``dg_mixture_covariance``: the result must equal
the one context's ``dg_covariance`` bit for bit where the per-density
arithmetic does not depend on the density's index (FP64; FP32 with
round-to-nearest), and the oracle's mixture aggregation within the path's
tolerance.  A second test runs ``multi.sharded_covariance`` in two processes
(gloo ranks) that share this GPU; their kernels never wait on each other.
"""
import datetime
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1907_06191_gb300 as dg  # noqa: E402


def _problem(p=3, m=5):
    rng = np.random.default_rng(404)
    act = (rng.random((37, 40)) > 0.3).astype(np.uint8)
    h, x0, y0 = 0.2, 0.5, -3.0
    src = []
    while len(src) < m:
        ex, ey = int(rng.integers(8, 32)), int(rng.integers(8, 29))
        if act[ey, ex]:
            src.append((x0 + (ex + rng.uniform(0.1, 0.9)) * h, y0 + (ey + rng.uniform(0.1, 0.9)) * h))
    return act, h, x0, y0, np.array(src)


KW = dict(D=2.0, sigma0=0.25)


def _ctx(p, prec, rnd, act, h, x0, y0):
    s = dg.DGSolver(p=p, precision=prec, device=0, rounding=rnd, **KW)
    s.set_geometry_mask(act, h, x0, y0)
    return s


@pytest.mark.parametrize("prec,rnd", [(dg.DG_FP64, dg.DG_ROUND_NEAREST),
                                      (dg.DG_FP32, dg.DG_ROUND_NEAREST),
                                      (dg.DG_FP32, dg.DG_ROUND_STOCHASTIC)])
@pytest.mark.parametrize("split", [[2, 3], [1, 1, 3]])
def test_mixture_covariance_of_split_contexts(prec, rnd, split):
    p = 3
    act, h, x0, y0, src = _problem(p)
    mesh = O.Mesh(p=p, active=act, h=h, x0=x0, y0=y0, k0=KW["D"])
    nsteps, dt = 70, 0.85 * O.rk3_real_limit() / O.power_rho(mesh)
    with _ctx(p, prec, rnd, act, h, x0, y0) as a:
        a.set_sources(src)
        a.step(nsteps, dt)
        s_all, mu_all, mass_all = a.covariance()
    moms, mom0s, lo = [], [], 0
    for k in split:
        with _ctx(p, prec, rnd, act, h, x0, y0) as b:
            b.set_sources(src[lo:lo + k])
            mom0s.append(b.moments())
            b.step(nsteps, dt)
            moms.append(b.moments())
        lo += k
    with _ctx(p, prec, rnd, act, h, x0, y0) as c:  # any context forms the mixture
        s_mix, mu_mix = c.mixture_covariance(np.concatenate(moms), np.concatenate(mom0s))
    if rnd == dg.DG_ROUND_NEAREST:
        assert np.array_equal(s_mix, s_all) and np.array_equal(mu_mix, mu_all)
    # the oracle's densities and mixture aggregation
    f0 = [O.init_gaussian(mesh, x, y, KW["sigma0"]) for x, y in src]
    mom0 = np.array([O.moments(mesh, f, x, y) for f, (x, y) in zip(f0, src)])
    mom = np.array([O.moments(mesh, O.rk3(mesh, f, nsteps, dt), x, y) for f, (x, y) in zip(f0, src)])
    s_ref, mu_ref, _ = O.aggregate(mom, mom0)
    tol = 1e-10 if prec == dg.DG_FP64 else 1e-5
    assert np.abs(s_mix - s_ref).max() < tol * np.abs(s_ref).max()
    assert np.abs(mass_all - mom[:, 0]).max() < tol * np.abs(mom[:, 0]).max()


def test_mixture_covariance_rejects_bad_arguments():
    act, h, x0, y0, src = _problem()
    with _ctx(3, dg.DG_FP64, dg.DG_ROUND_NEAREST, act, h, x0, y0) as c:
        with pytest.raises(dg.DgError) as ei:
            c.mixture_covariance(np.zeros((0, 6)), np.zeros((0, 6)))
        assert ei.value.code == dg.DG_EINVAL


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q, nsteps, dt):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    try:
        import torch.distributed as dist
        import paper_1907_06191_gb300 as dgl
        from paper_1907_06191_gb300.multi import sharded_covariance
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=60))
        act, h, x0, y0, src = _problem()
        with dgl.DGSolver(p=3, precision=dgl.DG_FP64, device=0, **KW) as s:
            s.set_geometry_mask(act, h, x0, y0)
            out = sharded_covariance(s, src, lambda c: c.step(nsteps, dt))
        q.put((rank, "ok", out))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error", repr(e)))


def test_sharded_covariance_two_ranks_on_this_gpu():
    """multi.sharded_covariance end to end: two gloo ranks, each with its own
    context on cuda:0, one gather of the moments, Sigma on each rank's device
    equal bit for bit to the one-context dg_covariance."""
    act, h, x0, y0, src = _problem()
    mesh = O.Mesh(p=3, active=act, h=h, x0=x0, y0=y0, k0=KW["D"])
    nsteps, dt = 40, 0.85 * O.rk3_real_limit() / O.power_rho(mesh)
    with _ctx(3, dg.DG_FP64, dg.DG_ROUND_NEAREST, act, h, x0, y0) as a:
        a.set_sources(src)
        a.step(nsteps, dt)
        s_all, mu_all, _ = a.covariance()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q, nsteps, dt)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        r, status, payload = q.get(timeout=300)
        res[r] = (status, payload)
    for p in procs:
        p.join(timeout=60)
    for r in range(2):
        status, payload = res[r]
        assert status == "ok", payload
        s3, mu, mom, mom0 = payload
        assert mom.shape == (len(src), 6)
        assert np.array_equal(s3, s_all) and np.array_equal(mu, mu_all)
