"""Replica bookkeeping of the multi-GPU benchmark.  A single system does not
shard without a per-panel exchange, so N GPUs run N independent replicas:
rank r solves its own system (seed 42 + r), no collective touches the data
path, the step time is the maximum over ranks (all ranks start together
after a barrier), and the throughput counts every rank's solve (weak
scaling).  Host logic only: the collective here is one scalar all-reduce of
the measured time (NCCL on the GPU machine, gloo in the CPU tests)."""
from __future__ import annotations

import os


def env():
    """(rank, world size, local rank) from the launcher's environment (1 process when unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def system_seed(rank: int) -> int:
    """Seed of the synthetic system that rank solves (each replica its own)."""
    return 42 + rank


def max_over_ranks(ms: float, dist=None, device="cpu") -> float:
    """The step time of the whole job: the largest of the ranks' times."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_tflops(world: int, flops_per_solve: float, ms: float) -> float:
    """Whole-job throughput: every rank's solve over the slowest rank's time."""
    return world * flops_per_solve / (ms * 1e-3) / 1e12
