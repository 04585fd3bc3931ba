"""Start points sharded across ranks (one process per GPU).

The densities of the Sigma scheme (Sec. 4.1) are independent: each rank
propagates a contiguous block of start points on its own copy of the
geometry, with no exchange during the time loop.  The only exchange is one
all-gather of the per-density raw moments ([m_r][6] FP64) after the last
step; the mixture covariance of the gathered moments is then formed on the
device by ``dg_mixture_covariance``.
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
    """All-gather the [m_r][6] moment blocks of every rank into [m_total][6]
    in rank order (torch.distributed; gloo on CPU tensors or nccl on CUDA
    tensors).  Blocks are padded to the largest shard for the collective."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    sizes = [shard(m_total, r, world).stop - shard(m_total, r, world).start
             for r in range(world)]
    assert local.shape == (sizes[rank], 6)
    width = max(sizes)
    buf = torch.zeros((width, 6), dtype=torch.float64, device=device)
    buf[:sizes[rank]] = torch.from_numpy(np.ascontiguousarray(local, dtype=np.float64)).to(buf.device)
    outs = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(outs, buf, group=group)
    return np.concatenate([o[:n].cpu().numpy() for o, n in zip(outs, sizes)], axis=0)
