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

import os

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


def closeness_checkpointed(partial, n: int, path: str, first: int = 0, count: int | None = None,
                           chunk: int = 16 * 1024):
    """All-source (or a source range's) distance sums, resumable.

    Runs the sources [first, first + count) in chunks of `chunk` sources
    through partial(first, count) -> (far, reach) (``Graph.closeness_range``
    or any callable returning int64 n-vectors), adds each chunk into running
    int64 sums and, after every chunk, saves the sums and the next source id
    to `path` (written to a temporary file, then renamed, so a crash leaves
    either the previous or the new checkpoint).  A call that finds `path`
    resumes after its last completed chunk; a checkpoint of another n or
    range raises ValueError.  Since far and reach are sums over sources, the
    resumed result equals an uninterrupted run bit for bit.  Returns (far,
    reach) as int64 numpy arrays; the checkpoint is left in place."""
    if count is None:
        count = n - first
    if first < 0 or count < 0 or first + count > n:
        raise ValueError("source range outside [0, n)")
    if chunk <= 0:
        raise ValueError("chunk must be positive")
    end = first + count
    far = np.zeros(n, np.int64)
    reach = np.zeros(n, np.int64)
    nxt = first
    if os.path.exists(path):
        with np.load(path) as ck:
            if int(ck["n"]) != n or int(ck["first"]) != first or int(ck["end"]) != end:
                raise ValueError(f"checkpoint {path} belongs to another graph or source range")
            far[:] = ck["far"]
            reach[:] = ck["reach"]
            nxt = int(ck["next"])
    while nxt < end:
        c = min(chunk, end - nxt)
        f, r = partial(nxt, c)
        far += np.asarray(f.cpu() if hasattr(f, "cpu") else f, dtype=np.int64)
        reach += np.asarray(r.cpu() if hasattr(r, "cpu") else r, dtype=np.int64)
        nxt += c
        tmp = path + ".tmp.npz"
        np.savez(tmp, n=n, first=first, end=end, next=nxt, far=far, reach=reach)
        os.replace(tmp, path)
    return far, reach
