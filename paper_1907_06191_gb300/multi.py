"""Start points sharded across ranks (one process per GPU).

The densities of the Sigma scheme (Sec. 4.1) are independent: each rank
propagates a contiguous block of start points on its own copy of the
geometry, with no exchange during the time loop.  The only exchange is one
all-gather of the per-density raw moments (at t and at 0, [m_r][12] FP64)
after the last step; the mixture covariance of the gathered moments is then
formed on the device by ``dg_mixture_covariance``.
"""
from __future__ import annotations

import numpy as np


def shard(m_total: int, rank: int, world: int) -> slice:
    """Contiguous block of start points owned by ``rank``: sizes differ by at
    most one, lower ranks take the remainder."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, rem = divmod(m_total, world)
    lo = rank * base + min(rank, rem)
    return slice(lo, lo + base + (1 if rank < rem else 0))


def gather_moments(local: np.ndarray, m_total: int, group=None, device=None) -> np.ndarray:
    """All-gather the [m_r][k] moment blocks of every rank into [m_total][k]
    in rank order (torch.distributed; gloo on CPU tensors or nccl on CUDA
    tensors).  Blocks are padded to the largest shard for the collective."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    sizes = [shard(m_total, r, world).stop - shard(m_total, r, world).start
             for r in range(world)]
    local = np.asarray(local, dtype=np.float64)
    k = local.shape[1] if local.ndim == 2 else 6
    local = local.reshape(-1, k)
    assert local.shape[0] == sizes[rank]
    width = max(sizes)
    buf = torch.zeros((width, k), dtype=torch.float64, device=device)
    if sizes[rank]:
        buf[:sizes[rank]] = torch.from_numpy(np.ascontiguousarray(local)).to(buf.device)
    outs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return np.concatenate([o[:n].cpu().numpy() for o, n in zip(outs, sizes)], axis=0)


def sharded_covariance(solver, sources, advance, group=None, device=None):
    """Sigma of all ``sources`` ([m_total, 2] start points) with the densities
    sharded across the ranks of ``group``.

    ``solver`` is this rank's context with its geometry already set (every
    rank the same geometry); ``advance(solver)`` carries its densities to the
    diffusion time (``solver.propagate_to(delta)`` or ``solver.step(n, dt)``;
    the step plan depends only on the geometry, so every rank takes the same
    one).  Each rank starts its own block, records the raw moments at 0 and
    at the end, and the blocks are gathered once (one collective of
    [m_r][12]).  Every rank then forms Sigma(Delta) - Sigma(0) of the whole
    mixture with ``dg_mixture_covariance``; the result does not depend on the
    number of ranks.  A rank whose block is empty (fewer start points than
    ranks) only takes part in the gather.

    Returns (sigma3, mu2, moments [m_total, 6], moments at 0 [m_total, 6]).
    """
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    sources = np.asarray(sources, dtype=np.float64).reshape(-1, 2)
    m_total = sources.shape[0]
    mine = sources[shard(m_total, rank, world)]
    if mine.shape[0]:
        solver.set_sources(mine)
        mom0 = solver.moments()
        advance(solver)
        mom = solver.moments()
        local = np.concatenate([mom, mom0], axis=1)
    else:
        local = np.zeros((0, 12))
    both = gather_moments(local, m_total, group=group, device=device)
    mom, mom0 = both[:, :6], both[:, 6:]
    s3, mu = solver.mixture_covariance(mom, mom0)
    return s3, mu, mom, mom0
