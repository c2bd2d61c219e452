"""Host-side logic for running the benchmark as N independent replicas (one process per
GPU, launched by torchrun): each rank holds its own copy of the graph and answers its own
queries; there is no data-path collective. The collectives here only synchronise timing
(barrier, max of the per-rank times) and add up the work done, so that the reported rate
is (units processed by all ranks) / (slowest rank's time).
"""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 if absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str) -> tuple[int, int, int]:
    """Join the process group when running with more than one rank."""
    world, rank, local = env()
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def _tensor(x, device):
    import torch
    return torch.tensor([float(x)], dtype=torch.float64, device=device)


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, device="cpu") -> float:
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = _tensor(x, device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device="cpu") -> float:
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = _tensor(x, device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def rank_slice(items, rank: int, world: int):
    """This rank's disjoint share of a common list (round-robin); shares cover the list."""
    return items[rank::world]


def aggregate_rate(units_all_ranks: float, slowest_ms: float) -> float:
    """Whole-job rate in units per second."""
    return units_all_ranks / (slowest_ms / 1e3) if slowest_ms > 0 else 0.0
