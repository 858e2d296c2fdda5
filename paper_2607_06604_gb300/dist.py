"""Host-side helpers for runs with one process per GPU.

The query path needs no collective on its data path: ranks either count
independent catalogues (a mock ensemble) or disjoint hub shards of one
catalogue (gs_options.shard / shards, the hub-window decomposition of Sec. 4.7).
The only exchanges are these reductions of finished results.
"""
from __future__ import annotations


def reduce_counts(t, group=None):
    """Sum integer histograms over ranks, exactly (int64 all-reduce).

    Counts are below 2^63, so the uint64 histogram travels as int64 bit
    patterns and comes back as uint64. Returns a new tensor.
    """
    import torch
    import torch.distributed as dist
    x = t.to(torch.int64) if t.dtype != torch.int64 else t.clone()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
    return x.to(t.dtype) if t.dtype != torch.int64 else x


def reduce_timing(ms: float, work: float, device=None, group=None):
    """(max over ranks of the timed milliseconds, sum over ranks of the work)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(w.item())


def shard_bounds(prefix, shards: int):
    """Contiguous ranges [lo, hi) of equal share of a nondecreasing prefix
    array (length n + 1), the rule the library applies to its row offsets."""
    import numpy as np
    prefix = np.asarray(prefix)
    n = len(prefix) - 1
    total = int(prefix[n])
    cuts = [0]
    for k in range(1, shards):
        target = total * k // shards
        cuts.append(int(np.searchsorted(prefix[:n], target, side="left")))
    cuts.append(n)
    return [(cuts[k], cuts[k + 1]) for k in range(shards)]
