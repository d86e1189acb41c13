"""Host-side multi-process helpers (one process per GPU).

Augmenting a batch has no data exchange between volumes: each volume has its
own transform, noise stream and loss, so several GPUs simply take disjoint
sets of volumes (the paper splits a batch evenly over its GPUs, Sec. 6.B).
The only collectives are the timing barrier and a max/sum over ranks.
"""
from __future__ import annotations

import os
from typing import Sequence

import torch
import torch.distributed as dist


def env_rank_world():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def init_from_env(backend: str = "nccl"):
    """Initialise the default process group from torchrun's environment
    (no-op for a single process).  Returns (rank, world, local_rank)."""
    rank, world, local = env_rank_world()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world, local


def barrier():
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def reduce_max(value: float, device="cpu") -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value: float, device="cpu") -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_noise_ids(n_local: int, rank: int):
    """Philox volume words (descriptor noise_id) of the n_local volumes of one
    replica: rank r takes r * n_local .. r * n_local + n_local - 1, so no two
    volumes of a multi-GPU job draw the same noise stream."""
    return [rank * n_local + b for b in range(n_local)]


def partition(weights: Sequence[int], world: int, rank: int):
    """Indices of the volumes rank `rank` of `world` takes: contiguous ranges
    with (nearly) equal total weight (e.g. output voxels).  Every index goes to
    exactly one rank; ranks keep the batch order."""
    n = len(weights)
    total = float(sum(weights))
    bounds = [0]
    acc, r = 0.0, 1
    for i, w in enumerate(weights):
        acc += w
        while r < world and acc >= total * r / world and len(bounds) <= r:
            bounds.append(i + 1)
            r += 1
    while len(bounds) < world:
        bounds.append(n)
    bounds.append(n)
    return list(range(bounds[rank], bounds[rank + 1]))
