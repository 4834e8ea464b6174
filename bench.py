"""Benchmark: single-source BFS throughput (GTEPS, harmonic mean over seeded
sources) of the BVSS path on one GB300, with its HBM roofline fraction.

One "step" = one BFS from each of the workload's seeded sources (the whole
hot path: level init, every level, un-permute).  Timing: CUDA events on the
stream the kernels run on, W >= 3 warm-up steps, barrier + synchronize
around the timed region, max over ranks.  The BVSS arrays of the bench
graphs are gigabytes (far larger than the 129 MB L2), so no separate L2
flush is done between timed iterations.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl blest|reference]

--impl reference times the CPU oracle (serial FIFO BFS) on a bounded sample
of the same workload and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import graphgen as gg  # noqa: E402

WORKLOADS = {
    # name: (builder, build options, description)
    "rmat24": (lambda: gg.rmat(24, 16, seed=2), dict(reorder=0),
               "RMAT scale 24 (16.7M vertices), edge factor 16, a=.57 b=c=.19, undirected, "
               "labels scrambled"),
    "rmat22": (lambda: gg.rmat(22, 16, seed=3), dict(reorder=0),
               "RMAT scale 22 (4.2M vertices), edge factor 16, undirected, labels scrambled"),
    "rmat16": (lambda: gg.rmat(16, 16, seed=1), dict(reorder=0),
               "RMAT scale 16 (65,536 vertices), edge factor 16, undirected, no reordering"),
    "grid4096": (lambda: gg.grid(4096, 4096, 0.05, 0.001, seed=2), dict(reorder=0),
                 "4096x4096 4-neighbour grid, 5% edges deleted, 0.1% random shortcuts"),
}
NUM_SOURCES = 64


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(log, n: int, reached: int) -> float:
    """Bytes one BFS must move, from the engine's per-level log (one pass over
    each array it touches; no credit for caching):
      top-down level: |Q| * 649 B (512 rowIds + 128 masks + 4 virtualToReal +
        4 queue entry + 1 frontier byte);
      lazy / bottom-up level: stage 2 reads V_curr and V_next (8 B per 32
        vertices) and writes V_curr and F for changed words (8 B per new vertex
        at most); bottom-up stage 1 reads V_curr and the in-neighbour mask
        (8 B per 32 vertices), two row pointers per probed vertex (16 B) and
        4 B per in-neighbour id read;
      every newly visited vertex: its level (4 B) and its degree (4 B);
      init: 4 B per vertex of levels and 5 bitvectors (20 B per 32 vertices)."""
    W = (n + 31) // 32
    b = 4.0 * n + 20.0 * W + 8.0 * reached
    for i, rec in enumerate(log):
        mode = rec["mode"]
        new = log[i + 1]["frontier"] if i + 1 < len(log) else 0
        if mode in (0, 1, 2, 3):
            b += rec["queue"] * 649.0
        if mode in (2, 3, 4):
            b += 8.0 * W + 8.0 * min(new, W)
        if mode == 4:
            b += 8.0 * W + 16.0 * rec.get("scanned_vertices", 0) + 4.0 * rec.get("scanned_arcs", 0)
    return b


def harmonic(x):
    x = np.asarray(x, np.float64)
    return float(len(x) / np.sum(1.0 / x))


def run_reference(args, rank, world):
    """CPU oracle on a bounded sample of the workload (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    build_fn, _, desc = WORKLOADS[args.workload]
    g = build_fn()
    srcs = gg.sources(g, NUM_SOURCES, 7)
    edges = []
    times = []
    budget = float(os.environ.get("BLEST_REF_BUDGET_S", "20"))
    t_all = time.perf_counter()
    k = 0
    for step in range(args.warmup + args.steps):
        s = int(srcs[k % len(srcs)])
        k += 1
        t0 = time.perf_counter()
        lv = oracle.bfs(g, s)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            edges.append(oracle.gteps_edges(g, lv))
        if time.perf_counter() - t_all > budget and len(times) >= 1:
            break
    rates = [e / t / 1e9 for e, t in zip(edges, times)]
    v = harmonic(rates)
    line = {"metric": "GTEPS (harm. mean/source), single-source BFS", "value": v, "unit": "GTEPS",
            "impl": "reference", "n_gpus": world, "steps": len(times), "warmup": args.warmup,
            "ms_per_step": float(np.mean(times) * 1e3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload, "graph": desc, "n": g.n, "nnz": g.nnz,
                       "sources": "seeded vertices of nonzero degree"},
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"{len(times)} single-source serial BFS runs (one step = one source)"},
            "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(g, srcs, budget_s=15.0):
    import oracle
    rates = []
    t_all = time.perf_counter()
    for s in srcs:
        t0 = time.perf_counter()
        lv = oracle.bfs(g, int(s))
        dt = time.perf_counter() - t0
        rates.append(oracle.gteps_edges(g, lv) / dt / 1e9)
        if time.perf_counter() - t_all > budget_s:
            break
    return {"value": harmonic(rates), "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"{len(rates)} of the workload's sources, one serial FIFO BFS each on one host core"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--impl", default="blest", choices=["blest", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sources", type=int, default=NUM_SOURCES)
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-policy arm")
    ap.add_argument("--block", type=int, default=0, help="CTA size override (256, 512, 1024)")
    ap.add_argument("--batch", type=int, default=0, help="VSSs in flight per warp override (1, 2, 4)")
    ap.add_argument("--levels", action="store_true", help="print the per-level log of the first source to stderr")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "blest" else args.warmup

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl" if args.impl == "blest" else "gloo")

    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return

    import torch
    import paper_2606_05081_gb300 as blest
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    build_fn, bopts, desc = WORKLOADS[args.workload]
    t0 = time.time()
    g = build_fn()
    gen_s = time.time() - t0
    # replicas: each rank runs its own seeded sources on its own copy (weak scaling)
    srcs = gg.sources(g, args.sources, 7 + rank)
    deg = np.diff(g.row_ptr)
    rp_d = torch.from_numpy(g.row_ptr).to(dev)
    col_d = torch.from_numpy(g.col).to(dev)
    if args.block:
        bopts = dict(bopts, block_threads=args.block)
    if args.batch:
        bopts = dict(bopts, vss_batch=args.batch)
    h = blest.build(g.n, rp_d, col_d, **bopts)
    del rp_d, col_d
    info = h.info()
    # a dedicated stream: the events below and the library's kernels share it
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    h.set_stream(stream.cuda_stream, True)
    out = torch.empty(g.n, dtype=torch.int32, device=dev)
    deg_d = torch.from_numpy(deg).to(dev)

    # edges per source (Graph500 convention: arcs out of reached vertices / 2)
    edges = []
    logs = []
    for s in srcs:
        h.bfs(int(s), out)
        h.sync()
        reached = out >= 0
        e = int(deg_d[reached].sum().item())
        edges.append(e if g.directed else e // 2)
        logs.append((h.level_log(), int(reached.sum().item())))
    if args.levels and rank == 0:
        for rec in logs[0][0]:
            print("level", json.dumps(rec), file=sys.stderr)

    starts = [torch.cuda.Event(enable_timing=True) for _ in srcs]
    ends = [torch.cuda.Event(enable_timing=True) for _ in srcs]

    def step(record):
        for i, s in enumerate(srcs):
            if record:
                starts[i].record(stream)
            h.bfs(int(s), out)
            if record:
                ends[i].record(stream)

    def measure(policy, engine_tc):
        """Warm-up, then the timed steps under one level-mode policy; returns
        per-source device ms [steps, sources], the timed region's ms and the
        per-source level logs of the policy."""
        h.set_engine(engine_tc)
        h.set_policy(policy)
        for _ in range(args.warmup):
            step(False)
        h.sync()
        torch.cuda.synchronize()
        psm = np.zeros((args.steps, len(srcs)))
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for k in range(args.steps):
            step(True)
            torch.cuda.synchronize()
            for i in range(len(srcs)):
                psm[k, i] = starts[i].elapsed_time(ends[i])
        t_end.record(stream)
        torch.cuda.synchronize()
        h.sync()
        if dist:
            dist.barrier()
        tot = t_start.elapsed_time(t_end)
        if dist:
            tt = torch.tensor([tot], device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            tot = float(tt.item())
        plogs = []
        for s_ in srcs:
            h.bfs(int(s_), out)
            h.sync()
            plogs.append(h.level_log())
        return psm, tot, plogs

    def gteps(psm):
        rates = (np.asarray(edges)[None, :] / (psm * 1e-3)) / 1e9
        v = harmonic(rates.ravel())
        if dist:
            vt = torch.tensor([v], device=dev, dtype=torch.float64)
            dist.all_reduce(vt)
            v = float(vt.item())
        return v

    from paper_2606_05081_gb300 import switch
    weights = switch.load_weights()
    policies = [("plain_tc", blest.POLICY_HEURISTIC, True), ("heuristic_cc", blest.POLICY_HEURISTIC, False)]
    if weights is not None and not args.no_learned:
        h.load_model(weights)
        policies.append(("learned", blest.POLICY_LEARNED, False))
    results = {}
    with ClockSampler(local) as clk:
        for name, pol, tc in policies:
            results[name] = measure(pol, tc)
    head = "learned" if "learned" in results else "heuristic_cc"
    per_source_ms, total_ms, head_logs = results[head]
    value = gteps(per_source_ms)
    variants = {name: {"gteps": gteps(r[0]), "per_source_ms_median": float(np.median(r[0])),
                       "ms_per_step": r[1] / args.steps} for name, r in results.items()}

    # roofline of the persistent BFS kernel under the headline policy
    hbm, peak_kind = peaks()
    mean_ms = per_source_ms.mean(axis=0)
    reached = [lg_r for _, lg_r in logs]
    alg = np.array([algorithmic_bytes(lg, g.n, r) for lg, r in zip(head_logs, reached)])
    achieved = float(np.sum(alg) / np.sum(mean_ms * 1e-3) / 1e9)
    logs = [(lg, r) for lg, r in zip(head_logs, reached)]

    # end to end through the C ABI with host buffers (synchronous calls)
    h.set_stream(None, False)
    host_out = torch.empty(g.n, dtype=torch.int32).pin_memory()
    host_np = host_out.numpy()
    e2e_rates = []
    for s, e in zip(srcs, edges):
        t0 = time.perf_counter()
        h.bfs(int(s), host_np)
        dt = time.perf_counter() - t0
        e2e_rates.append(e / dt / 1e9)
    e2e = harmonic(e2e_rates)

    line = {
        "metric": "GTEPS (harm. mean/source), single-source BFS", "value": value, "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "graph": desc, "n": g.n, "nnz": int(info["nnz"]),
                   "sources": len(srcs), "reorder": int(info["reorder"]), "lazy": int(info["lazy"]),
                   "switching": int(info["switching"]), "policy": head,
                   "udiv": info["update_divergence"], "num_vss": int(info["num_vss"]),
                   "block_threads": int(info["block_threads"]), "grid_blocks": int(info["grid_blocks"]),
                   "vss_batch": int(bopts.get("vss_batch", 2)),
                   "l2": "inputs larger than L2 (BVSS arrays), no flush", "parallelism": f"replicas{world}",
                   "graph_gen_s": round(gen_s, 1), "build_ms": round(info["build_ms"], 1)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "peak_kind": peak_kind,
                     "kernel": "k_bfs (persistent, all levels)"},
        "e2e": {"value": e2e, "unit": "GTEPS", "h2d_bytes_per_step": 4 * len(srcs),
                "d2h_bytes_per_step": 4 * g.n * len(srcs)},
        "gpu_launches": args.steps * len(srcs) * len(results),
        "variants": variants,
        "clocks": clk.summary(),
        "per_source_ms_median": float(np.median(per_source_ms)),
        "levels_source0": [[r["mode"], r["queue"], round(r["t_ns"] / 1e3, 1)] for r in logs[0][0]],
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, srcs)
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
