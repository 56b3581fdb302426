"""Independent replicas on several GPUs, one process per GPU.

Markov chains and their samples are independent (Sec. 2.2.5: the sampler runs
many chains, and NetKet spreads them over MPI processes), so each rank advances
its own chains and its own copy of the parameters with no data-path exchange:
weak scaling.  What the ranks do share is host-side bookkeeping: distinct chain
seeds, barriers around the timed region, the maximum of the ranks' times, and
the whole-job rate computed from it.
"""
import os

import torch
import torch.distributed as dist


def env_world():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(world: int, backend: str) -> None:
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)


def barrier(world: int) -> None:
    if world > 1:
        dist.barrier()


def replica_seed(seed: int, rank: int) -> int:
    """Chain seed of a rank: distinct per rank, rank 0 keeps the workload's seed."""
    return seed + 7919 * rank


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The largest value of x over all ranks (the job's time is its slowest rank's)."""
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds
