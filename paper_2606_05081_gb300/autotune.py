"""Autotuner for the single-source kernel.

Two levels, both timed as whole BFSs with CUDA events on tuning sources
the caller keeps disjoint from the ones it measures:

* ``autotune(h, ...)`` tunes the launch of one handle: CTA size (256, 512,
  1024 threads), VSS passes a warp keeps in flight in top-down levels
  (1, 2, 4) and, on the sigma = 8, tau = 128 layout only, the top-down
  hit-test engine (b1 MMA of Fig. 3 or CUDA cores) -- unless the handle
  runs the learned policy with weights loaded, which picks the engine per
  level itself, so the engine setting would not change what runs;
* ``autotune_layout(build, ...)`` builds the graph once per BVSS layout --
  slice width sigma in {8, 16, 32} with its warp-wide VSS (tau = 32 *
  32 / sigma), plus the narrow tau = 32 VSS at sigma = 8 -- tunes each
  launch, keeps the fastest handle and closes the others.
"""
from __future__ import annotations

import itertools

from . import POLICY_LEARNED

BLOCKS = (256, 512, 1024)
BATCHES = (1, 2, 4)
LAYOUTS = ((8, 128), (8, 32), (16, 64), (32, 32))


def autotune(h, sources, reps: int = 2, stream=None):
    import torch
    dev = torch.device("cuda")
    out = torch.empty(h.n, dtype=torch.int32, device=dev)
    s = stream if stream is not None else torch.cuda.Stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    info = h.info()
    learned = info["policy"] == POLICY_LEARNED and info["model_loaded"]
    engines = (False, True) if (info["sigma"], info["tau"]) == (8, 128) and not learned else (bool(info["engine_tc"]),)
    results = []
    with torch.cuda.stream(s):
        h.set_stream(s.cuda_stream, True)
        for blk, bat, tc in itertools.product(BLOCKS, BATCHES, engines):
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


def autotune_layout(build, sources, layouts=LAYOUTS, reps: int = 2, stream=None):
    """build(sigma, tau) -> a configured handle (policy and weights set).
    Returns (fastest handle, its tuning record with per-layout results)."""
    best_h, best, per = None, None, []
    for sigma, tau in layouts:
        h = build(sigma, tau)
        r = autotune(h, sources, reps=reps, stream=stream)
        r.update(sigma=sigma, tau=tau)
        per.append({"sigma": sigma, "tau": tau, "ms_per_bfs": round(r["ms_per_bfs"], 4),
                    "block_threads": r["block_threads"], "vss_batch": r["vss_batch"], "engine_tc": r["engine_tc"]})
        if best is None or r["ms_per_bfs"] < best["ms_per_bfs"]:
            if best_h is not None:
                best_h.close()
            best_h, best = h, r
        else:
            h.close()
    best["layouts"] = per
    return best_h, best
