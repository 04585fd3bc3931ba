"""Start points sharded across ranks (gloo, CPU processes).

The densities of the Sigma scheme (Sec. 4.1) are independent, so ranks
propagate disjoint blocks of start points and exchange only the per-density
moments once.  Here each rank runs its block on the CPU oracle; the gathered
moments must equal the unsharded run bit for bit, and a rank that dies before
the exchange must surface as an error on the survivor, not a hang.
"""
import datetime
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_1907_06191_gb300.multi import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _problem():
    import oracle as O
    rng = np.random.default_rng(31)
    act = (rng.random((14, 16)) > 0.2).astype(np.uint8)
    mesh = O.Mesh(p=2, active=act, h=0.4, k0=1.0)
    src = []
    while len(src) < 7:
        ex, ey = int(rng.integers(3, 13)), int(rng.integers(3, 11))
        if act[ey, ex]:
            src.append(((ex + 0.5) * 0.4, (ey + 0.5) * 0.4))
    return mesh, np.array(src)


def _moments_for(mesh, src, nsteps=6, dt=0.004):
    import oracle as O
    out = []
    for x, y in src:
        u = O.rk3(mesh, O.init_gaussian(mesh, x, y, 0.3), nsteps, dt)
        out.append(O.moments(mesh, u, x, y))
    return np.array(out).reshape(-1, 6)


def _worker(rank, world, port, q, fail_rank):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_1907_06191_gb300.multi import gather_moments
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=8))
        mesh, src = _problem()
        mine = src[shard(len(src), rank, world)]
        mom = _moments_for(mesh, mine)
        if rank == fail_rank:
            os._exit(3)  # dies between steps, before the exchange
        allm = gather_moments(mom, len(src))
        q.put((rank, "ok", allm))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error", repr(e)))


def _run(world, fail_rank=-1, timeout=120):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, fail_rank)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    expect = world - (1 if fail_rank >= 0 else 0)
    for _ in range(expect):
        r, status, payload = q.get(timeout=timeout)
        res[r] = (status, payload)
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return res, [p.exitcode for p in procs]


def test_shard_partition():
    for m in (1, 5, 64, 65, 127):
        for world in (1, 2, 3, 8):
            parts = [shard(m, r, world) for r in range(world)]
            assert parts[0].start == 0 and parts[-1].stop == m
            for a, b in zip(parts, parts[1:]):
                assert a.stop == b.start
            sizes = [p.stop - p.start for p in parts]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_moments_equal_unsharded_bitwise(world):
    import oracle as O
    O.build()
    mesh, src = _problem()
    ref = _moments_for(mesh, src)
    res, codes = _run(world)
    for r in range(world):
        status, allm = res[r]
        assert status == "ok", allm
        assert np.array_equal(allm, ref)
    s_ref = O.aggregate(ref, ref)[0]
    assert np.array_equal(O.aggregate(res[0][1], ref)[0], s_ref)


def test_dead_rank_is_reported_not_hung():
    import oracle as O
    O.build()
    res, codes = _run(2, fail_rank=1)
    assert codes[1] == 3
    status, payload = res[0]
    assert status == "error"


class _OracleSolver:
    """Stand-in for one rank's DGSolver on the CPU: the same four calls
    sharded_covariance makes, answered by the oracle."""

    def __init__(self, mesh, nsteps=6, dt=0.004):
        self.mesh, self.nsteps, self.dt = mesh, nsteps, dt
        self.src, self.u = None, None

    def set_sources(self, xy):
        import oracle as O
        self.src = np.asarray(xy).reshape(-1, 2)
        self.u = [O.init_gaussian(self.mesh, x, y, 0.3) for x, y in self.src]

    def moments(self):
        import oracle as O
        return np.array([O.moments(self.mesh, u, x, y) for u, (x, y) in zip(self.u, self.src)])

    def advance(self):
        import oracle as O
        self.u = [O.rk3(self.mesh, u, self.nsteps, self.dt) for u in self.u]

    def mixture_covariance(self, mom, mom0):
        import oracle as O
        s3, mu, _ = O.aggregate(mom, mom0)
        return s3, mu


def _sigma_worker(rank, world, port, q, m):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    from paper_1907_06191_gb300.multi import sharded_covariance
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world,
                                timeout=datetime.timedelta(seconds=20))
        mesh, src = _problem()
        s3, mu, mom, mom0 = sharded_covariance(_OracleSolver(mesh), src[:m],
                                               lambda s: s.advance())
        q.put((rank, "ok", (s3, mu, mom, mom0)))
        dist.destroy_process_group()
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error", repr(e)))


@pytest.mark.parametrize("world,m", [(2, 7), (3, 7), (3, 2)])
def test_sharded_covariance_equals_unsharded(world, m):
    """The host side of the sharded Sigma: start points split over gloo
    ranks, raw moments at 0 and at t gathered in one collective, Sigma of the
    whole mixture on every rank.  It must equal the unsharded aggregation bit
    for bit, also when a rank owns no start point (m = 2 < 3 ranks)."""
    import oracle as O
    O.build()
    mesh, src = _problem()
    ref = _OracleSolver(mesh)
    ref.set_sources(src[:m])
    mom0 = ref.moments()
    ref.advance()
    mom = ref.moments()
    s_ref, mu_ref, _ = O.aggregate(mom, mom0)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sigma_worker, args=(r, world, port, q, m)) for r in range(world)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(world):
        r, status, payload = q.get(timeout=120)
        res[r] = (status, payload)
    for p in procs:
        p.join(timeout=30)
    for r in range(world):
        status, payload = res[r]
        assert status == "ok", payload
        s3, mu, gm, gm0 = payload
        assert np.array_equal(gm, mom) and np.array_equal(gm0, mom0)
        assert np.array_equal(s3, s_ref) and np.array_equal(mu, mu_ref)
