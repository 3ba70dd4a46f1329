"""Host-side sharding of independent eigenproblems across ranks.

Each (lattice, Bloch vector) problem is independent (one eigenproblem per
wave vector along a band path), so ranks split the problem list with no
collective on the data path.  The only collectives are host-side: gathering
eigenvalues at the end and the max-over-ranks / sum-over-ranks bookkeeping of
the benchmark.
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Round-robin share of ``items`` for ``rank`` of ``world`` (contiguous order kept)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return [x for i, x in enumerate(items) if i % world == rank]


def shard_indices(count: int, rank: int, world: int):
    return shard(list(range(count)), rank, world)


def reduce_timing(elapsed_ms: float, work: float, group=None, device=None):
    """(max elapsed over ranks, sum of work over ranks) with torch.distributed, if initialised."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return elapsed_ms, work
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(w.item())


def gather_results(local: dict, group=None):
    """Gather {problem index: eigenvalue list} from every rank onto every rank (host objects)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return dict(local)
    out = [None] * dist.get_world_size(group)
    dist.all_gather_object(out, local, group=group)
    merged = {}
    for part in out:
        merged.update(part)
    return merged
