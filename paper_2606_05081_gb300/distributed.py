"""Closeness centrality split across processes (one per GPU).

All-source closeness (§6.2) is a sum over sources: far[u] = sum_s d(s, u)
and reach[u] = #{s : d(s, u) finite} on an undirected graph (Eq. 6), so the
sources partition into contiguous ranges, each rank runs the multi-source
BFS batches of its own range (``Graph.closeness_range``) with no exchange
during the traversal, and one integer sum of the two n-vectors over the
ranks completes the result; cc[u] = (reach[u] - 1) / far[u] (Eq. 7 with the
component-size normalisation) is then computed in fp64 on every rank.
"""
from __future__ import annotations

import numpy as np


def source_ranges(n: int, world: int):
    """Contiguous source ranges, one per rank, sizes differing by at most one
    batch of 1024 (the multi-source BFS batch width) so every rank runs whole
    batches except possibly the last."""
    batches = (n + 1023) // 1024
    per, extra = divmod(batches, world)
    out, b = [], 0
    for r in range(world):
        nb = per + (1 if r < extra else 0)
        first = min(n, b * 1024)
        last = min(n, (b + nb) * 1024)
        out.append((first, last - first))
        b += nb
    return out


def closeness_allreduce(partial, n: int, rank: int, world: int, dist=None, group=None):
    """partial(first, count) -> (far, reach): this rank's sums over its
    sources (int64 n-vectors, numpy or torch).  Returns the summed far and
    reach (int64 numpy) and cc (float64 numpy), identical on every rank."""
    import torch
    first, count = source_ranges(n, world)[rank]
    far, reach = partial(first, count)
    far_t = torch.as_tensor(np.asarray(far.cpu() if hasattr(far, "cpu") else far, dtype=np.int64))
    reach_t = torch.as_tensor(np.asarray(reach.cpu() if hasattr(reach, "cpu") else reach, dtype=np.int64))
    if dist is not None and world > 1:
        dist.all_reduce(far_t, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(reach_t, op=dist.ReduceOp.SUM, group=group)
    f = far_t.numpy()
    r = reach_t.numpy()
    cc = np.zeros(n, np.float64)
    nz = f > 0
    cc[nz] = (r[nz] - 1).astype(np.float64) / f[nz].astype(np.float64)
    return f, r, cc
