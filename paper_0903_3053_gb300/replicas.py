"""Host-side logic of replica runs over several GPUs (one process per GPU).

Chains are independent Markov chains, so a run over N GPUs is N replicas of the
same parameter points, each with its own Philox chain ids (the paper ran one
parameter point per GPU, up to eight per host, Sec. 3).  No chain data crosses
ranks: the process group only carries the start/stop barrier and the
max-over-ranks time.  The backend is whatever the caller initialised (NCCL on
GPUs; gloo on the host for the tests).
"""
from __future__ import annotations

import os

CHAIN_ID_STRIDE = 1 << 16  # chain ids of rank r: [r * stride, (r + 1) * stride)


def env_world() -> tuple[int, int, int]:
    """(world, rank, local_rank) from the torchrun environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def chain_id(rank: int, index: int) -> int:
    """Philox chain id of replica `index` on `rank`; ranks never share a stream."""
    if not 0 <= index < CHAIN_ID_STRIDE:
        raise ValueError(f"replica index {index} out of range")
    cid = rank * CHAIN_ID_STRIDE + index
    if cid >= 1 << 32:
        raise ValueError(f"rank {rank} too large for 32-bit chain ids")
    return cid


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Units processed by the whole job."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank: float, seconds: float, world: int, device: str = "cuda") -> float:
    """Whole-job throughput: units all ranks processed / the slowest rank's time."""
    return sum_over_ranks(units_per_rank, world, device) / max_over_ranks(seconds, world, device)
