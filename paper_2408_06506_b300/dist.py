"""Multi-GPU bookkeeping for the tactile step: one process per GPU, envs sharded.

Environments are independent (no exchange step), so N ranks split the envs into
contiguous shards and run the step on their own shard with no collective on the data
path.  The only cross-rank operations of the step are the barriers around a timed region
and the max-over-ranks reduction of its duration.  The calibration workload (gradient
descent on the contact and shading parameters) has one real exchange: the gradient of a
parameter that every shard shares (the per-pixel shading coefficients, or contact
parameters given once for all envs) is the sum of the shards' gradients, one all-reduce
per step.  These helpers work with any torch.distributed backend (nccl on GPUs, gloo on
CPU for tests).
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


def sum_shared_grads(tensors, dist=None) -> None:
    """Sum, in place and over all ranks, the gradients of parameters every rank's shard
    shares (identity without a process group or with one rank).  The tensors are
    flattened into one buffer per dtype and device so that a step makes one collective
    per buffer; None entries are skipped."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return
    import torch
    groups = {}
    for t in tensors:
        if t is not None:
            groups.setdefault((t.dtype, t.device), []).append(t)
    for ts in groups.values():
        flat = torch.cat([t.reshape(-1) for t in ts])
        dist.all_reduce(flat, op=dist.ReduceOp.SUM)
        o = 0
        for t in ts:
            n = t.numel()
            t.copy_(flat[o:o + n].view_as(t))
            o += n
