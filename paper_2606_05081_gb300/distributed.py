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


def _as_int64_tensor(x, device):
    """An int64 torch tensor of x (numpy or torch) on `device`."""
    import torch
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.int64)
    return torch.as_tensor(np.asarray(x, dtype=np.int64), device=device)


def reduce_device(dist, group=None):
    """The device the all-reduce of the sums must run on: the current CUDA
    device for a NCCL group (NCCL reduces device memory only), the host for
    gloo and the other CPU backends."""
    import torch
    if dist is not None and dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def closeness_allreduce(partial, n: int, rank: int, world: int, dist=None, group=None):
    """partial(first, count) -> (far, reach): this rank's sums over its
    sources (int64 n-vectors, numpy or torch, host or device).  The two
    vectors are summed over the ranks in place -- on the GPU when the group
    is NCCL, on the host for gloo -- and the result is returned as int64
    numpy far and reach and float64 numpy cc, identical on every rank."""
    first, count = source_ranges(n, world)[rank]
    far, reach = partial(first, count)
    dev = reduce_device(dist if world > 1 else None, group)
    far_t = _as_int64_tensor(far, dev)
    reach_t = _as_int64_tensor(reach, dev)
    if dist is not None and world > 1:
        dist.all_reduce(far_t, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(reach_t, op=dist.ReduceOp.SUM, group=group)
    f = far_t.cpu().numpy()
    r = reach_t.cpu().numpy()
    cc = np.zeros(n, np.float64)
    nz = f > 0
    cc[nz] = (r[nz] - 1).astype(np.float64) / f[nz].astype(np.float64)
    return f, r, cc


def graph_fingerprint(row_ptr, col) -> str:
    """A fingerprint of a CSR graph (n, arc count and a SHA-256 of both
    arrays), stored in closeness checkpoints so a checkpoint is never merged
    into the sums of another graph."""
    import hashlib
    rp = np.ascontiguousarray(np.asarray(row_ptr.cpu() if hasattr(row_ptr, "cpu") else row_ptr, dtype=np.int64))
    cl = np.ascontiguousarray(np.asarray(col.cpu() if hasattr(col, "cpu") else col, dtype=np.int32))
    h = hashlib.sha256()
    h.update(rp.tobytes())
    h.update(cl.tobytes())
    return f"n={len(rp) - 1};arcs={len(cl)};sha256={h.hexdigest()}"


def closeness_checkpointed(partial, n: int, path: str, first: int = 0, count: int | None = None,
                           chunk: int = 16 * 1024, fingerprint: str = ""):
    """All-source (or a source range's) distance sums, resumable.

    Runs the sources [first, first + count) in chunks of `chunk` sources
    through partial(first, count) -> (far, reach) (``Graph.closeness_range``
    or any callable returning int64 n-vectors), adds each chunk into running
    int64 sums and, after every chunk, saves the sums and the next source id
    to `path` (written to a temporary file, then renamed, so a crash leaves
    either the previous or the new checkpoint).  A call that finds `path`
    resumes after its last completed chunk.  The checkpoint records n, the
    range and `fingerprint` (``graph_fingerprint`` of the CSR); one whose
    record differs from the call's raises ValueError instead of being
    merged.  Since far and reach are sums over sources, the
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
            stored = str(ck["fingerprint"]) if "fingerprint" in ck.files else ""
            if stored != fingerprint:
                raise ValueError(f"checkpoint {path} belongs to another graph "
                                 f"(fingerprint {stored!r}, expected {fingerprint!r})")
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
        np.savez(tmp, n=n, first=first, end=end, next=nxt, far=far, reach=reach, fingerprint=fingerprint)
        os.replace(tmp, path)
    return far, reach
