"""Replicas with read sharding (multi-GPU host logic).

The search path shards by reads: every rank (one process per GPU) holds its own replica of
the index and searches its own batch of reads, so nothing is exchanged on the data path.  Only
the timing is reduced (the slowest rank bounds the job), and results may optionally be
gathered to rank 0.  Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env_rank():
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's read batch: distinct per rank, equal to the base seed on rank 0."""
    return base_seed + 1000 * rank


def shard_range(n: int, world: int, rank: int):
    """[start, end) of rank's share when one batch of n items is split across ranks."""
    per = (n + world - 1) // world
    s = min(n, rank * per)
    return s, min(n, s + per)


def _device():
    if dist.is_initialized() and dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(x: float) -> float:
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier():
    if dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def job_throughput(units_per_rank: int, seconds_per_rank: float) -> float:
    """Whole-job throughput: units every rank processed / the slowest rank's time."""
    total = sum_over_ranks(float(units_per_rank))
    return total / max_over_ranks(seconds_per_rank)


def gather_counts(counts: torch.Tensor):
    """Per-query interval counts of every rank, on rank 0 (list of CPU tensors), else None."""
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return [counts.cpu()]
    dev = _device()
    n = torch.tensor([counts.numel()], dtype=torch.int64, device=dev)
    sizes = [torch.zeros_like(n) for _ in range(dist.get_world_size())]
    dist.all_gather(sizes, n)
    mx = int(max(s.item() for s in sizes))
    buf = torch.zeros(mx, dtype=counts.dtype, device=dev)
    buf[:counts.numel()] = counts.to(dev)
    out = [torch.zeros(mx, dtype=counts.dtype, device=dev) for _ in sizes]
    dist.all_gather(out, buf)
    if dist.get_rank() != 0:
        return None
    return [o[:int(s.item())].cpu() for o, s in zip(out, sizes)]
