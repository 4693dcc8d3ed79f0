"""Sharding over ranks (one process per GPU, torch.distributed).

Imaging: instances are independent, so each rank images a contiguous block of frames and no
data crosses ranks (weak scaling; only timings are max-reduced).

Gradient imaging of one sky image from many channels: chi2 and its gradient are sums over
visibilities, so each rank holds the visibilities of a block of channels and the per-rank
loss and gradient are summed with one all-reduce per step -- the only data exchange.

Every helper is a no-op in a single process (torch.distributed not initialised or one rank).
"""
from __future__ import annotations

import torch


def rank_world() -> tuple[int, int]:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def block(n: int, rank: int, world: int) -> slice:
    """Contiguous share of n items for `rank` of `world`; shares differ by at most one item."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("block: need 0 <= rank < world and n >= 0")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return slice(lo, lo + q + (1 if rank < r else 0))


def all_sum_(t: torch.Tensor) -> torch.Tensor:
    """In-place sum over ranks."""
    import torch.distributed as dist
    if rank_world()[1] > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def all_max(x: float, device="cpu") -> float:
    """Largest value over ranks (timings: the job is as slow as its slowest rank)."""
    import torch.distributed as dist
    if rank_world()[1] == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
