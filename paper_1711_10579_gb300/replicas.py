"""Replica runs over several GPUs.

A single Newton solve does not shard (it would need a domain decomposition of
the grid), but independent scenarios and requests do: each rank solves its own
scenarios on its own GPU with no data exchange.  Only the timing is combined:
the job's time is the slowest rank's, and its throughput counts every rank's
converged solves.
"""
from __future__ import annotations


def scenario_seed(base: int, rank: int) -> int:
    """Seed of a rank's scenarios, so replicas solve different ones."""
    return base + 7919 * rank


def aggregate(local_ms: float, local_converged: int, dist=None):
    """(solves/s of the whole job, slowest rank's ms, total converged).

    ``dist`` is an initialised torch.distributed module or None for one
    process; the reductions are a MAX of the times and a SUM of the counts.
    """
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_converged / (local_ms * 1e-3), local_ms, local_converged
    import torch

    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    n = torch.tensor([local_converged], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    ms, total = float(t.item()), int(n.item())
    return total / (ms * 1e-3), ms, total
