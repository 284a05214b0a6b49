"""Process-group helpers of the multi-GPU bench.

One process per GPU, launched by torch.distributed.run (RANK, WORLD_SIZE,
LOCAL_RANK and MASTER_* from the environment). The contraction workload
shards over independent units (specs, samples, states) with no exchange, so
every rank runs its own copy of the per-GPU workload on its own seeded data
(weak scaling) and the only collective is one all-reduce of a scalar: the
slowest rank's time.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def env() -> tuple[int, int, int]:
    """(rank, world size, local rank); (0, 1, 0) outside a launched job."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str) -> None:
    """Joins the process group when the job has more than one rank."""
    _, world, _ = env()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)


def barrier() -> None:
    if dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float, device: torch.device | str = "cpu") -> float:
    """The largest x over all ranks (x itself with one rank)."""
    if not dist.is_initialized():
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, ms_max: float, world: int) -> float:
    """Whole-job throughput: every rank processed units_per_rank in at most ms_max."""
    return world * units_per_rank / (ms_max * 1e-3)


def data_seed(base: int, rank: int) -> int:
    """Seed of a rank's own synthetic operands."""
    return base * 1000 + rank


def finish() -> None:
    if dist.is_initialized():
        dist.destroy_process_group()
