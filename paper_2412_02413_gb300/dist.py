"""Multi-GPU host logic. Frames are independent, so the AS-TAX path shards by
frame with no data-path collective (weak scaling). The only collectives are
a barrier and a max over the ranks' timings.

Each process drives one GPU. RANK, LOCAL_RANK and WORLD_SIZE come from the
launcher (torchrun).
"""
from __future__ import annotations

import os
from typing import List, Tuple


def env_rank() -> Tuple[int, int, int]:
    """(rank, local_rank, world_size) from the launcher environment."""
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, local, world


def shard_frames(n_total: int, rank: int, world: int) -> List[int]:
    """Round-robin frame indices of one rank: frame f goes to rank f mod world."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    return list(range(rank, n_total, world))


def init(backend: str) -> bool:
    """Initialise torch.distributed when WORLD_SIZE > 1. Returns True if it did."""
    import torch.distributed as dist
    _, _, world = env_rank()
    if world <= 1:
        return False
    if not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend)
    return True


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (x itself when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def finalize():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()
