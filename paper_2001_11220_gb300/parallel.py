"""Multi-GPU use: one process per GPU, no collective on the data path.

A single grid's step has no exchange between independent GPUs here (every
line solve needs the whole line), so several GPUs run replicas or shards of
an ensemble: instances are independent problems, split in contiguous blocks
across ranks.  The only collectives are for measurement (max over ranks of
the timed region, sum of the work done).
"""
from __future__ import annotations


def shard(ninst: int, world: int, rank: int) -> range:
    """Contiguous block of instance indices owned by rank (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(ninst, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def aggregate(local_ms: float, local_units: float, group=None):
    """(max over ranks of local_ms, sum over ranks of local_units, throughput = units / max seconds)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local_ms, local_units, local_units / (local_ms / 1e3)
    backend = dist.get_backend(group)
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    ms, units = float(t.item()), float(u.item())
    return ms, units, units / (ms / 1e3)
