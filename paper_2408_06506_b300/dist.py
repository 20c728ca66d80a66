"""Multi-GPU bookkeeping for the tactile step: one process per GPU, envs sharded.

Environments are independent (no exchange step), so N ranks split the envs into
contiguous shards and run the step on their own shard with no collective on the data
path.  The only cross-rank operations are the barriers around a timed region and the
max-over-ranks reduction of its duration.  These helpers work with any
torch.distributed backend (nccl on GPUs, gloo on CPU for tests).
"""
from __future__ import annotations


def env_shard(n_envs: int, rank: int, world: int) -> tuple:
    """Contiguous env range [lo, hi) of `rank`; sizes differ by at most one."""
    if world < 1 or not (0 <= rank < world) or n_envs < 0:
        raise ValueError(f"bad shard request: n_envs={n_envs} rank={rank} world={world}")
    base, extra = divmod(n_envs, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of a per-rank float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
