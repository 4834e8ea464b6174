"""Autotuner for the single-source kernel's launch shape.

Tries every combination of CTA size (256, 512, 1024 threads), VSSs a warp
keeps in flight in top-down levels (1, 2, 4) and the top-down hit-test
engine (b1 MMA or CUDA cores), timing whole BFSs with CUDA events on
tuning sources the caller keeps disjoint from the ones it measures, and
leaves the handle on the fastest.  The slice width is fixed at sigma = 8
(the Fig. 3 tensor-core layout and the BVSS lane mapping are sigma = 8).
"""
from __future__ import annotations

import itertools

import numpy as np

BLOCKS = (256, 512, 1024)
BATCHES = (1, 2, 4)
ENGINES = (False, True)


def autotune(h, sources, reps: int = 2, stream=None):
    import torch
    dev = torch.device("cuda")
    out = torch.empty(h.n, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.Stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with torch.cuda.stream(s):
        h.set_stream(s.cuda_stream, True)
        for blk, bat, tc in itertools.product(BLOCKS, BATCHES, ENGINES):
            h.set_launch(blk, bat)
            h.set_engine(tc)
            for src in sources[:2]:          # warm-up
                h.bfs(int(src), out)
            h.sync()
            ev0.record(s)
            for _ in range(reps):
                for src in sources:
                    h.bfs(int(src), out)
            ev1.record(s)
            torch.cuda.synchronize()
            h.sync()
            results.append((ev0.elapsed_time(ev1) / (reps * len(sources)), blk, bat, tc))
        h.set_stream(None, False)
    results.sort()
    best = results[0]
    h.set_launch(best[1], best[2])
    h.set_engine(best[3])
    return {"ms_per_bfs": best[0], "block_threads": best[1], "vss_batch": best[2], "engine_tc": int(best[3]),
            "tried": [[round(r[0], 4), r[1], r[2], int(r[3])] for r in results]}
