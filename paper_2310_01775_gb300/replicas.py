"""Independent replicas over ranks: the host side of the multi-GPU runs.

The planning path shards by instance: every rank (one process per GPU)
solves its own seeded problem, with no collective on the data path.  The
only exchange is the timing: the slowest rank's time over the timed steps
(max-reduced), from which the whole-job throughput is all ranks' units
divided by that time.  NCCL on GPUs, gloo on host-only runs.
"""
from __future__ import annotations

import os

import torch


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str | None = None) -> tuple[int, int, int]:
    """Join the process group when there is more than one rank."""
    world, rank, local = env()
    if world > 1 and not torch.distributed.is_initialized():
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        torch.distributed.init_process_group(backend)
    return world, rank, local


def rank_seed(base: int, rank: int) -> int:
    """Each rank's problem seed: disjoint scenes and noise per replica."""
    return base + 1000 * rank


def max_over_ranks(x: float, device=None) -> float:
    """The largest x of all ranks (x itself on one rank)."""
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (ms_max / 1e3)


def barrier() -> None:
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()


def finish() -> None:
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.destroy_process_group()
