"""Rank utilities for running frames on several GPUs of one node (one process per GPU).

Views are independent units of the removal effect (Section IV-B sums dSE over views), so a
multi-GPU run shards views across ranks and needs no collective on the data path.  The one
exchange the method has -- adding the per-splat dMSE_k / I_k partials of all ranks before a
pruning decision -- is ``ordered_sum``: gather, then add in rank order, so the result is the
same bits whatever the arrival order.  Everything here works with the gloo backend on CPU.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env_ranks() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (defaults: single process)."""
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, local, world


def init(backend: str) -> None:
    _, _, world = env_ranks()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)


def active() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def barrier() -> None:
    if active():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (x itself on one rank)."""
    if not active():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    if not active():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_range(n_items: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous block of items for ``rank``; sizes differ by at most one, earlier ranks larger."""
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def ordered_sum(local: torch.Tensor) -> torch.Tensor:
    """Sum of ``local`` over ranks, added in rank order 0, 1, ... (deterministic)."""
    if not active():
        return local.clone()
    parts = [torch.empty_like(local) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, local.contiguous())
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out
