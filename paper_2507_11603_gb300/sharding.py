"""Photon sharding across ranks (one process per GPU).

Photon packets are independent given the geometry (THOR Sec. 3.6.2-3.6.3 replicate
subvolumes and balance photon counts); every photon's random stream is keyed by its
global id, so a photon's history does not depend on the rank that runs it.  Rank r of
W therefore runs the contiguous id range returned by ``photon_range`` and the integer
tallies of all ranks sum exactly to those of a single-rank run.  The only exchange is
that final sum (``merge_counts``), outside any timed region.
"""
from __future__ import annotations


def photon_range(rank: int, world: int, n_per_rank: int, base: int = 0):
    """Weak scaling: rank r runs ids [base + r n, base + (r + 1) n)."""
    if not (0 <= rank < world) or n_per_rank <= 0:
        raise ValueError("need 0 <= rank < world and n_per_rank > 0")
    first = base + rank * n_per_rank
    return first, n_per_rank


def split_range(rank: int, world: int, n_total: int, base: int = 0):
    """Strong scaling: a fixed total split into contiguous, nearly equal id ranges."""
    if not (0 <= rank < world) or n_total < 0:
        raise ValueError("need 0 <= rank < world and n_total >= 0")
    q, r = divmod(n_total, world)
    first = base + rank * q + min(rank, r)
    return first, q + (1 if rank < r else 0)


def merge_counts(counts, group=None):
    """Sum integer spectra / tallies over ranks in place (torch.distributed all-reduce)."""
    import torch
    import torch.distributed as dist
    t = counts if isinstance(counts, torch.Tensor) else torch.as_tensor(counts)
    t = t.to(torch.int64)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def merge_weights(hist, n_local: int, group=None):
    """Reweighted spectra (Sec. 5.1 post-processing) over ranks: each rank's histogram is a
    sum of weights divided by its own photon count n_local; the merged result is the sum of
    the weights over all ranks divided by the total count (FP64 all-reduce)."""
    import torch
    import torch.distributed as dist
    t = torch.as_tensor(hist, dtype=torch.float64) * float(n_local)
    n = torch.tensor([float(n_local)], dtype=torch.float64)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(n, op=dist.ReduceOp.SUM, group=group)
    return t / n

