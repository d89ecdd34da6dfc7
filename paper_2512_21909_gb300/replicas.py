"""Multi-GPU bookkeeping: replicas only.

One gradient runs on one GPU.  With N processes (one per GPU, launched by
torchrun) every rank works on its own systems; nothing on the data path is
exchanged.  torch.distributed is used only for the timing barrier, the
max-over-ranks of measured times and gathering small per-rank results.
"""
from __future__ import annotations

import os


def init(backend: str | None = None):
    """(rank, world size); initialises torch.distributed when WORLD_SIZE > 1
    (NCCL when CUDA is available, else gloo)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            if backend is None:
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
    return rank, world


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x: float, world: int) -> float:
    """Maximum of a scalar over ranks (identity for one rank)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(items, rank: int, world: int):
    """Round-robin share of independent work items for this rank."""
    return [it for k, it in enumerate(items) if k % world == rank]


def finalize(world: int):
    if world > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()
