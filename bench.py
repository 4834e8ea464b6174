"""Benchmark of the BVSS BFS path on one GB300: throughput (GTEPS,
harmonic mean over seeded sources) with its HBM roofline fraction, for every
configuration of the workload set, each checked against the CPU oracle.

Headline (the JSON line's `value`): single-source BFS, 64 seeded sources on
each of two graphs --
  * RMAT scale 24, edge factor 16 (16.7M vertices), JaccardWithWindows
    reordering with W = 2^16;
  * a 4096 x 4096 road-like grid (4-neighbour, 5 % of edges deleted, 0.1 %
    random shortcuts), RCM reordering.
One "step" = one BFS from every source of every graph (the whole hot path:
level init, every level, un-permute into the caller's ids).

Arms, each timed over the same steps:
  plain  the paper's method: hand-set rule (lazy/eager by U_div, Eq. 5
         switch), b1 MMA hit test, default launch shape;
  tuned  the learned level-mode policy with the autotuned launch shape
         (the headline `value`), falling back to the rule on the CUDA-core
         engine when no trained weights are present.
Timing: CUDA events on the stream the kernels run on, W >= 3 warm-up steps,
synchronize around the timed region, max over ranks.  The BVSS arrays are
gigabytes (far larger than the 129 MB L2), so no separate L2 flush is done.

With no --workload, the line also carries `per_config`: one entry per
configuration (C1 RMAT 16 plain; C2 the headline; C3 multi-source BFS on
RMAT 22 with 64 / 256 / 1024 lanes, the 10,000-graph Barabasi-Albert batch
and learned + batched against plain single-source on the same graph and
sources; C4 all-source closeness on RMAT 18 and the 2048^2 grid; C5 the
learned policy on held-out families), each with its roofline and a
`levels_bit_exact` count taken outside the timed regions against the CPU
oracle on all host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl blest|reference]

--impl reference times the CPU oracle (serial FIFO BFS) on a bounded sample
of the headline workload and prints the same JSON line with
"impl": "reference".
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

REORDER_RCM, REORDER_JACCARD = 1, 2
GRAPHS = {
    "rmat24_jaccard": (lambda: gg.rmat(24, 16, seed=2), dict(reorder=REORDER_JACCARD, jaccard_window=65536),
                       "RMAT scale 24, edge factor 16, a=.57 b=c=.19, undirected, scrambled labels, "
                       "JaccardWithWindows W=65536"),
    "grid4096_rcm": (lambda: gg.grid(4096, 4096, 0.05, 0.001, seed=2), dict(reorder=REORDER_RCM),
                     "4096x4096 4-neighbour grid, 5% edges deleted, 0.1% random shortcuts, RCM"),
    "rmat24": (lambda: gg.rmat(24, 16, seed=2), dict(reorder=0),
               "RMAT scale 24, edge factor 16, undirected, scrambled labels, no reordering"),
    "rmat22": (lambda: gg.rmat(22, 16, seed=3), dict(reorder=0),
               "RMAT scale 22, edge factor 16, undirected, scrambled labels, no reordering"),
    "rmat16": (lambda: gg.rmat(16, 16, seed=1), dict(reorder=0),
               "RMAT scale 16, edge factor 16, undirected, no reordering"),
}
WORKLOADS = {
    "all": ["rmat24_jaccard", "grid4096_rcm"],
    "sssp_pair": ["rmat24_jaccard", "grid4096_rcm"],
    "rmat24": ["rmat24"],
    "rmat22": ["rmat22"],
    "rmat16": ["rmat16"],
    "grid4096_rcm": ["grid4096_rcm"],
    "rmat24_jaccard": ["rmat24_jaccard"],
}
DEFAULT_WORKLOAD = "all"
# the other rows of the path, each with its own JSON line
EXTRA_WORKLOADS = ["msbfs_rmat22", "closeness_rmat18", "closeness_grid2048_part", "closeness_grid2048",
                   "bfs_many_ba10k", "switch_heldout", "ablation", "order_study", "msbfs_one"]
NUM_SOURCES = 64
METRIC = "GTEPS (harm. mean/source), single-source BFS"


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


def algorithmic_bytes(log, n: int, reached: int, sigma: int = 8, tau: int = 128) -> float:
    """Bytes one BFS must move, from the engine's per-level log (one pass over
    each array it touches; no credit for caching):
      top-down level: |Q| * (4 tau rowIds + 4 tau/theta mask words + 8 queue
        entry + sigma/8 frontier bytes), 649 B per VSS at sigma 8, tau 128;
      lazy / bottom-up level: stage 2 reads V_curr and V_next (8 B per 32
        vertices) and writes V_curr and F for changed words (8 B per new vertex
        at most); bottom-up stage 1 reads V_curr and the in-neighbour mask
        (8 B per 32 vertices), the 16-byte head (first four in-neighbours) of
        each probed vertex and 4 B per further in-neighbour id read;
      every newly visited vertex: its level (4 B) and its degree (4 B);
      init: 4 B per vertex of levels and 5 bitvectors (20 B per 32 vertices).
    The caller adds 12 B per vertex for the un-permute of a reordered graph
    (permutation entry, the gathered level, the stored level)."""
    W = (n + 31) // 32
    per_vss = 4.0 * tau + 4.0 * tau / (32 // sigma) + 8.0 + sigma / 8.0
    b = 4.0 * n + 20.0 * W + 8.0 * reached
    for i, rec in enumerate(log):
        mode = rec["mode"]
        new = log[i + 1]["frontier"] if i + 1 < len(log) else 0
        if mode in (0, 1, 2, 3):
            b += rec["queue"] * per_vss
        if mode in (2, 3, 4):
            b += 8.0 * W + 8.0 * min(new, W)
        if mode == 4:
            b += 8.0 * W + 16.0 * rec.get("scanned_vertices", 0) + 4.0 * rec.get("scanned_arcs", 0)
    return b


KERNEL_SOURCES = ["paper_2606_05081_gb300/csrc/bfs.cu", "paper_2606_05081_gb300/csrc/common.cuh",
                  "paper_2606_05081_gb300/csrc/mlp.h", "paper_2606_05081_gb300/csrc/handle.h"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_bfs_traffic.json")


MS_KERNEL_SOURCES = ["paper_2606_05081_gb300/csrc/msbfs.cu", "paper_2606_05081_gb300/csrc/tc.cuh",
                     "paper_2606_05081_gb300/csrc/common.cuh", "paper_2606_05081_gb300/csrc/handle.h"]


def kernel_sha(sources=None) -> str:
    import hashlib
    hsh = hashlib.sha256()
    for f in (sources or KERNEL_SOURCES):
        with open(os.path.join(ROOT, f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()[:16]


def measured_traffic(runs_layouts):
    """Per-launch DRAM bytes of k_bfs (dram__bytes_read.sum + dram__bytes_write.sum
    from ncu) for each (graph, sigma, tau) the step ran, averaged over its
    graphs; None when a record is missing or was taken on other kernel
    sources."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    d = json.load(open(TRAFFIC_FILE))
    if d.get("kernel_sha") != kernel_sha():
        return None
    recs = {(r["graph"], r["sigma"], r["tau"]): r["bytes_per_launch"] for r in d.get("records", [])}
    vals = [recs.get(k) for k in runs_layouts]
    if any(v is None for v in vals):
        return None
    return float(np.mean(vals))


def nvtx_range(name=None):
    """Open (name) or close (None) an NVTX range around a timed region, so a
    profiler can select exactly its launches (ncu --nvtx --nvtx-include
    "timed_tuned/"); a no-op where NVTX is unavailable."""
    try:
        import torch
        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def harmonic(x):
    x = np.asarray(x, np.float64)
    return float(len(x) / np.sum(1.0 / x))


def cpu_sample(g, srcs, budget_s):
    """The oracle (serial FIFO BFS, one host core) on a bounded sample."""
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
    return rates


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle (serial FIFO BFS, one host core) on
    the workload's graphs and seeded sources, rank 0 only.  A step is one
    oracle BFS per graph, step k taking each graph's source k (mod 64); W
    untimed warm-up steps, then K timed steps (stopped early only if the
    whole run passes BLEST_REF_BUDGET_S seconds, default 300)."""
    if rank != 0:
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "workload": args.workload,
                          "unavailable": "the reference arm times the single-source workloads; the oracle's "
                                         "multi-source, closeness and batched results are checked in tests/"}),
              flush=True)
        return
    import oracle
    names = WORKLOADS[args.workload]
    graphs = {nm: GRAPHS[nm][0]() for nm in names}
    srcs = {nm: gg.sources(g, NUM_SOURCES, 7) for nm, g in graphs.items()}
    cap = float(os.environ.get("BLEST_REF_BUDGET_S", "300"))

    def step(k):
        out = {}
        for nm, g in graphs.items():
            s = int(srcs[nm][k % len(srcs[nm])])
            t0 = time.perf_counter()
            lv = oracle.bfs(g, s)
            dt = time.perf_counter() - t0
            out[nm] = oracle.gteps_edges(g, lv) / dt / 1e9
        return out

    t_start = time.perf_counter()
    for w in range(args.warmup):
        step(w)
    rates = {nm: [] for nm in names}
    step_s = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        for nm, v in step(args.warmup + k).items():
            rates[nm].append(v)
        step_s.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > cap:
            break
    allr = [v for nm in names for v in rates[nm]]
    v = harmonic(allr)
    per_graph = {nm: {"gteps": harmonic(rates[nm]), "sources_timed": len(rates[nm])} for nm in names}
    line = {"metric": METRIC, "value": v, "unit": "GTEPS", "impl": "reference", "n_gpus": world,
            "steps": len(step_s), "warmup": args.warmup, "ms_per_step": float(np.mean(step_s)) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": args.workload, "graphs": {nm: GRAPHS[nm][2] for nm in names},
                       "sources": "64 seeded vertices of nonzero degree per graph; step k runs source k "
                                  "of each graph"},
            "per_graph": per_graph,
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": f"{len(step_s)} timed steps of one serial FIFO BFS per graph "
                                       f"({len(allr)} BFS runs) on one host core, after {args.warmup} "
                                       "untimed warm-up steps"},
            "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


class GraphRun:
    """One bench graph: the plain handle (default layout), the tuned handle
    (the autotuner's layout; the plain one when tuning is off), sources,
    edge counts and per-arm timings."""

    def __init__(self, name, args, rank, dev, torch, blest, stream):
        build_fn, bopts, desc = GRAPHS[name]
        self.name, self.desc, self.bopts = name, desc, bopts
        t0 = time.time()
        self.g = g = build_fn()
        self.gen_s = time.time() - t0
        self.srcs = gg.sources(g, args.sources, 7 + rank)
        self.tune_srcs = gg.sources(g, 8, 1000 + rank)
        rp_d = torch.from_numpy(g.row_ptr).to(dev)
        col_d = torch.from_numpy(g.col).to(dev)
        t0 = time.time()
        self.h = blest.build(g.n, rp_d, col_d, **bopts)
        self.build_s = time.time() - t0
        del rp_d, col_d
        self.h_tuned = self.h
        self.info = self.h.info()
        self.stream = stream
        self.h.set_stream(stream.cuda_stream, True)
        self.out = torch.empty(g.n, dtype=torch.int32, device=dev)
        deg_d = torch.from_numpy(np.diff(g.row_ptr)).to(dev)
        self.edges, self.reached = [], []
        for s in self.srcs:
            self.h.bfs(int(s), self.out)
            self.h.sync()
            r = self.out >= 0
            e = int(deg_d[r].sum().item())
            self.edges.append(e if g.directed else e // 2)
            self.reached.append(int(r.sum().item()))
        self.ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in self.srcs]

    def build_layout(self, blest, sigma, tau, weights, policy):
        h = blest.build(self.g.n, self.g.row_ptr, self.g.col, sigma=sigma, tau=tau, **self.bopts)
        if weights is not None:
            h.load_model(weights)
        h.set_policy(policy)
        return h

    def step(self, h, record):
        for i, s in enumerate(self.srcs):
            if record:
                self.ev[i][0].record(self.stream)
            h.bfs(int(s), self.out)
            if record:
                self.ev[i][1].record(self.stream)

    def logs(self, h):
        out = []
        for s in self.srcs:
            h.bfs(int(s), self.out)
            h.sync()
            out.append(h.level_log())
        return out

    def close(self):
        if self.h_tuned is not self.h:
            self.h_tuned.close()
        self.h.close()


class Ctx:
    """What every part of a bench run shares: torch, the binding, the device,
    the stream the library runs on, the trained weights, rank and world."""

    def __init__(self, args, rank, world, local, dist):
        import torch
        import paper_2606_05081_gb300 as blest
        from paper_2606_05081_gb300 import switch
        torch.cuda.set_device(local)
        self.torch, self.blest, self.dist = torch, blest, dist
        self.args, self.rank, self.world, self.local = args, rank, world, local
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.Stream(self.dev)
        torch.cuda.set_stream(self.stream)
        self.weights = switch.load_weights()
        self.hbm, self.peak_kind = peaks()

    def events(self):
        t = self.torch
        return t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)


def run_single_source(ctx, names, steps, warmup, tune=True, ablation=False, layout=None, launch=None,
                      levels=False, sources=NUM_SOURCES):
    """Plain and tuned single-source arms over `names` (GRAPHS keys): GTEPS,
    roofline of k_bfs, end to end through the C ABI, and levels_bit_exact
    of the tuned arm against the oracle.  Returns (fields of the JSON line,
    the GraphRun objects, still open)."""
    torch, blest, dist = ctx.torch, ctx.blest, ctx.dist
    from paper_2606_05081_gb300 import autotune
    rank, dev, stream = ctx.rank, ctx.dev, ctx.stream
    args_src = argparse.Namespace(sources=sources)
    runs = [GraphRun(nm, args_src, rank, dev, torch, blest, stream) for nm in names]
    weights = ctx.weights
    tuned_policy = blest.POLICY_LEARNED if weights is not None else blest.POLICY_HEURISTIC
    tune_info = {}
    for r in runs:
        if weights is not None:
            r.h.load_model(weights)
        if tune:
            r.h_tuned, tune_info[r.name] = autotune.autotune_layout(
                lambda sg, ta, r=r: r.build_layout(blest, sg, ta, weights, tuned_policy), r.tune_srcs, reps=3,
                stream=stream)
        elif layout:
            sg, ta = (int(x) for x in layout.split(","))
            r.h_tuned = r.build_layout(blest, sg, ta, weights, tuned_policy)
        if not tune and launch:
            bt, bb = (int(x) for x in launch.split(","))
            tune_info[r.name] = {"block_threads": bt, "vss_batch": bb, "engine_tc": 0, "fixed": True}
        r.h_tuned.set_stream(stream.cuda_stream, True)
        ti = tune_info.get(r.name, {})
        r.tuned = (int(ti.get("block_threads", 512)), int(ti.get("vss_batch", 2)), bool(ti.get("engine_tc", 0)))
        if levels and rank == 0:
            r.h_tuned.set_policy(tuned_policy)
            for rec in r.logs(r.h_tuned)[0]:
                print(r.name, "level", json.dumps(rec), file=sys.stderr)

    arms = {"plain": (blest.POLICY_HEURISTIC, "default", True), "tuned": (tuned_policy, "tuned", None)}
    if ablation:
        arms = {"plain": arms["plain"],
                "rule_cc": (blest.POLICY_HEURISTIC, "default", False),
                "rule_cc_tuned": (blest.POLICY_HEURISTIC, "tuned", False),
                "tuned": arms["tuned"]}

    def set_arm(r, arm):
        """The arm's handle, configured: plain = default layout and launch,
        the paper's rule with the b1 MMA hit test; tuned = the autotuner's
        layout and launch under the learned policy."""
        pol, lnch, tc = arms[arm]
        h = r.h if arm == "plain" else r.h_tuned
        if lnch == "default":
            h.set_launch(512, 2)
        else:
            h.set_launch(r.tuned[0], r.tuned[1])
        h.set_engine(r.tuned[2] if tc is None else tc)
        h.set_policy(pol)
        return h

    results = {}
    with ClockSampler(ctx.local) as clk:
        for arm in arms:
            for r in runs:
                h = set_arm(r, arm)
                for _ in range(warmup):
                    r.step(h, False)
                h.sync()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            t0e, t1e = ctx.events()
            psm = {r.name: np.zeros((steps, len(r.srcs))) for r in runs}
            t0e.record(stream)
            nvtx_range("timed_" + arm)
            for k in range(steps):
                for r in runs:
                    r.step(set_arm(r, arm), True)
                torch.cuda.synchronize()
                for r in runs:
                    for i in range(len(r.srcs)):
                        psm[r.name][k, i] = r.ev[i][0].elapsed_time(r.ev[i][1])
            nvtx_range()
            t1e.record(stream)
            torch.cuda.synchronize()
            for r in runs:
                r.h.sync()
                r.h_tuned.sync()
            if dist:
                dist.barrier()
            tot = t0e.elapsed_time(t1e)
            if dist:
                tt = torch.tensor([tot], device=dev)
                dist.all_reduce(tt, op=dist.ReduceOp.MAX)
                tot = float(tt.item())
            results[arm] = (psm, tot, {r.name: r.logs(set_arm(r, arm)) for r in runs})

    def gteps_of(psm_by_graph):
        rates = []
        per = {}
        for r in runs:
            rr = (np.asarray(r.edges)[None, :] / (psm_by_graph[r.name] * 1e-3)) / 1e9
            per[r.name] = harmonic(rr.ravel())
            rates.append(rr.ravel())
        v = harmonic(np.concatenate(rates))
        if dist:
            vt = torch.tensor([v], device=dev, dtype=torch.float64)
            dist.all_reduce(vt)
            v = float(vt.item())
        return v, per

    value, per_graph = gteps_of(results["tuned"][0])
    plain_value, plain_per = gteps_of(results["plain"][0])

    # roofline of the persistent BFS kernel under the headline arm
    hbm, peak_kind = ctx.hbm, ctx.peak_kind
    alg_b, dev_s = 0.0, 0.0
    per_graph_roof = {}
    for r in runs:
        logs = results["tuned"][2][r.name]
        ti = r.h_tuned.info()
        gb = sum(algorithmic_bytes(lg, r.g.n, rc, ti["sigma"], ti["tau"]) +
                 (12.0 * r.g.n if r.info["reorder"] else 0.0) for lg, rc in zip(logs, r.reached))
        gs = float(results["tuned"][0][r.name].mean(axis=0).sum()) * 1e-3
        alg_b += gb
        dev_s += gs
        per_graph_roof[r.name] = {"achieved_gbs": gb / gs / 1e9, "frac": gb / gs / 1e9 / hbm,
                                  "algorithmic_bytes_per_launch": gb / len(r.srcs),
                                  "traffic": measured_traffic([(r.name, ti["sigma"], ti["tau"])])}
    achieved = alg_b / dev_s / 1e9

    # end to end through the C ABI with host buffers, headline arm
    e2e_rates, d2h = [], 0
    for r in runs:
        h = set_arm(r, "tuned")
        h.set_stream(None, False)
        host = torch.empty(r.g.n, dtype=torch.int32).pin_memory().numpy()
        for s_, e in zip(r.srcs, r.edges):
            t0 = time.perf_counter()
            h.bfs(int(s_), host)
            e2e_rates.append(e / (time.perf_counter() - t0) / 1e9)
        d2h += 4 * r.g.n * len(r.srcs)
    e2e = harmonic(e2e_rates)

    # levels of every timed source of the tuned arm against the oracle (outside the timed regions)
    exact = {}
    for r in runs:
        h = set_arm(r, "tuned")
        h.set_stream(None, False)
        exact[r.name] = levels_exact_single(r.g, r.srcs, h, torch, dev)

    graphs_cfg = {}
    for r in runs:
        graphs_cfg[r.name] = {
            "graph": r.desc, "n": r.g.n, "nnz": int(r.info["nnz"]), "num_vss": int(r.info["num_vss"]),
            "udiv": round(r.info["update_divergence"], 1), "lazy": int(r.info["lazy"]),
            "switching": int(r.info["switching"]), "reorder": int(r.info["reorder"]),
            "gteps_tuned": per_graph[r.name], "gteps_plain": plain_per[r.name],
            "per_source_ms_median_tuned": float(np.median(results["tuned"][0][r.name])),
            "per_source_ms_median_plain": float(np.median(results["plain"][0][r.name])),
            "tuned_launch": {"block_threads": r.tuned[0], "vss_batch": r.tuned[1], "engine_tc": int(r.tuned[2]),
                             "sigma": int(r.h_tuned.info()["sigma"]), "tau": int(r.h_tuned.info()["tau"])},
            "graph_gen_s": round(r.gen_s, 1), "build_s": round(r.build_s, 2),
            "build_ms_device": round(r.info["build_ms"], 1),
            "levels_bit_exact": exact[r.name], "sources": len(r.srcs),
            "levels_source0_tuned": [[x["mode"], x["queue"], round(x["t_ns"] / 1e3, 1)]
                                     for x in results["tuned"][2][r.name][0]][:40]}
    line = {
        "value": value, "unit": "GTEPS",
        "ms_per_step": results["tuned"][1] / steps,
        "graphs": graphs_cfg,
        "plain": {"value": plain_value, "ms_per_step": results["plain"][1] / steps,
                  "what": "hand-set rule (U_div lazy/eager, Eq. 5 switch), b1 MMA hit test, default launch"},
        "speedup_vs_plain": value / plain_value,
        "levels_bit_exact": int(sum(exact.values())), "sources": int(sum(len(r.srcs) for r in runs)),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": measured_traffic([(r.name, r.h_tuned.info()["sigma"], r.h_tuned.info()["tau"])
                                                  for r in runs]), "peak_kind": peak_kind,
                     "kernel": "k_bfs (persistent, all levels)",
                     "algorithmic_bytes_per_launch": alg_b / sum(len(r.srcs) for r in runs),
                     "kernel_sha": kernel_sha(), "per_graph": per_graph_roof},
        "e2e": {"value": e2e, "unit": "GTEPS", "h2d_bytes_per_step": 4 * sum(len(r.srcs) for r in runs),
                "d2h_bytes_per_step": d2h},
        "gpu_launches": steps * sum(len(r.srcs) for r in runs),   # one k_bfs per BFS of the tuned arm
        "clocks": clk.summary(),
        "autotune": {k: {kk: vv for kk, vv in v.items() if kk != "tried"} for k, v in tune_info.items()},
    }
    if ablation:
        what = {"plain": "the paper's rule, b1 MMA hit test, sigma 8 / tau 128, 512-thread CTAs",
                "rule_cc": "the paper's rule, CUDA-core hit test, sigma 8 / tau 128, 512-thread CTAs",
                "rule_cc_tuned": "the paper's rule, CUDA-core hit test, autotuned layout and launch",
                "tuned": "learned per-level policy, autotuned layout and launch"}
        line["ablation"] = {}
        for arm in arms:
            v, per = gteps_of(results[arm][0])
            line["ablation"][arm] = {"value": v, "per_graph": per, "what": what[arm]}
    return line, runs


def levels_exact_single(g, srcs, h, torch, dev, chunk=16):
    """How many of the sources give a whole level array equal to the
    oracle's (one serial BFS per source, all host cores)."""
    import oracle
    out = torch.empty(g.n, dtype=torch.int32, device=dev)
    ok = 0
    for i in range(0, len(srcs), chunk):
        part = np.asarray(srcs[i:i + chunk])
        ref = oracle.bfs_many(g, part)
        for j, s_ in enumerate(part):
            h.bfs(int(s_), out)
            ok += int(np.array_equal(out.cpu().numpy(), ref[j]))
    return ok


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + EXTRA_WORKLOADS)
    ap.add_argument("--impl", default="blest", choices=["blest", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sources", type=int, default=NUM_SOURCES)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (tuned arm = default launch)")
    ap.add_argument("--levels", action="store_true", help="per-level log of the first source to stderr")
    ap.add_argument("--ablation", action="store_true",
                    help="also time the rungs between the plain and the tuned arm: the paper's rule with the "
                         "CUDA-core hit test on the default layout, then on the autotuned layout and launch")
    ap.add_argument("--tau", type=int, default=0, help="VSS width of the multi-source and closeness builds "
                    "(0 = 128)")
    ap.add_argument("--layout", default=None, help="sigma,tau of the tuned arm when the autotuner is off")
    ap.add_argument("--launch", default=None, help="block_threads,vss_batch of the tuned arm when the autotuner "
                    "is off")
    ap.add_argument("--scale", type=int, default=20, help="RMAT scale of the msbfs_one workload")
    ap.add_argument("--kappa", type=int, default=1024, help="sources of the msbfs_one workload")
    ap.add_argument("--engine", default="cc", choices=["cc", "tc"], help="multi-source stage 1 of msbfs_one")
    ap.add_argument("--direction", type=int, default=0, choices=[0, 1, 2],
                    help="multi-source stage 1 of msbfs_one: 0 push, 1 pull on dense levels, 2 pull")
    ap.add_argument("--staged", type=int, default=1, choices=[0, 1],
                    help="level output of msbfs_one: 1 staged bytes and a closing transpose, 0 direct stores")
    ap.add_argument("--configs", default="C1,C3,C4,C5",
                    help="per_config entries besides the headline (C2) of the default workload")
    args = ap.parse_args()

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
    args.warmup = max(args.warmup, 3)
    ctx = Ctx(args, rank, world, local, dist)
    if args.workload in EXTRA_WORKLOADS:
        run_extra(args, ctx)
        if dist:
            dist.destroy_process_group()
        return

    fields, runs = run_single_source(ctx, WORKLOADS[args.workload], args.steps, args.warmup,
                                     tune=not args.no_tune, ablation=args.ablation, layout=args.layout,
                                     launch=args.launch, levels=args.levels, sources=args.sources)
    line = {"metric": METRIC, "value": fields.pop("value"), "unit": fields.pop("unit"),
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": fields.pop("ms_per_step"), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": args.workload if args.workload != "all" else "sssp_pair (C2) + per_config",
                       "sources_per_graph": args.sources,
                       "policy": "learned+autotuned" if ctx.weights is not None else "heuristic+autotuned",
                       "l2": "inputs larger than L2 (BVSS arrays), no flush", "parallelism": f"replicas{world}",
                       "graphs": fields.pop("graphs")}}
    line.update(fields)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rates = []
        for r in runs:
            rates += cpu_sample(r.g, r.srcs, 12.0 / len(runs))
        line["cpu_baseline"] = {"value": harmonic(rates), "unit": "GTEPS", "cores": 1, "kind": "oracle",
                                "sample": f"{len(rates)} of the workload's sources (all graphs), one serial "
                                          "FIFO BFS each on one host core, about 12 s"}
    for r in runs:
        r.close()
    del runs
    if args.workload == "all":
        want = [c.strip() for c in args.configs.split(",") if c.strip()]
        per = {"C2": {"what": "single-source BFS, RMAT 24 (Jaccard) + 4096^2 grid (RCM), 64 sources each: "
                              "the headline fields of this line",
                      "value": line["value"], "plain": line["plain"]["value"], "unit": "GTEPS",
                      "roofline": line["roofline"], "levels_bit_exact": line["levels_bit_exact"],
                      "sources": line["sources"]}}
        t_all = time.time()
        with ClockSampler(local) as clk:
            for c in want:
                t0 = time.time()
                per[c] = PER_CONFIG[c](ctx)
                per[c]["wall_s"] = round(time.time() - t0, 1)
        per["clocks"] = clk.summary()
        per["wall_s"] = round(time.time() - t_all, 1)
        line["per_config"] = per
        if "C3" in per and "learned_batched_vs_plain" in per["C3"]:
            line["learned_batched_vs_plain"] = per["C3"]["learned_batched_vs_plain"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# ------------------------------------------------------------ byte models
def msbfs_algorithmic_bytes(st, n, tau=128, sigma=8, levels_out=True, closeness=False):
    """Bytes a multi-source call must move, from its work counters (one pass
    over each array touched, no credit for caching), per the terms of the
    multi-source path:
      stage 1, per processed VSS: its BVSS lane words (4 tau row ids +
        4 tau / theta mask words), its virtualToReal entry and queue entry
        (8 B), the kappa-bit frontier elements of its slice set's sigma
        vertices (sigma kappa / 8 B) and the set's active word (kappa / 8 B);
        4 B per nonzero 32-lane hit word OR-ed into V_next;
      stage 2, per dirty slice set: its sigma vertices' elements of V_next
        and V_curr read and of F and V_curr written (4 kappa / 8 B each);
      pulled levels: every vertex's V_curr element (kappa / 8 B) and, per
        in-neighbour read, its frontier element, slice-set stamp and id
        (kappa / 8 + 8 B);
      init: F, V_curr, V_next zeroed (3 kappa / 8 B per vertex) per launch;
      levels: the output floor, 4 kappa B per vertex per launch (each level
        written once);
      closeness: far and reach, 12 B per vertex per batch."""
    kappa = st["kappa"]
    theta = 32 // sigma
    per_vss = 4.0 * tau + 4.0 * tau / theta + 8.0 + sigma * kappa / 8.0 + kappa / 8.0
    b = st["vss"] * per_vss + 4.0 * st["hit_words"] + st["dirty_sets"] * sigma * 4.0 * kappa / 8.0
    b += st.get("pull_levels", 0) * n * kappa / 8.0 + st.get("pull_arcs", 0) * (kappa / 8.0 + 8.0)
    b += st["launches"] * n * 3.0 * kappa / 8.0
    if levels_out:
        b += st["launches"] * 4.0 * kappa * n
    if closeness:
        b += st["launches"] * 12.0 * n
    return b


def _roof(ctx, bytes_, seconds, kernel, traffic=None, **extra):
    a = bytes_ / seconds / 1e9
    d = {"bound": "hbm", "achieved": a, "peak": ctx.hbm, "unit": "GB/s", "frac": a / ctx.hbm,
         "traffic": traffic, "peak_kind": ctx.peak_kind, "kernel": kernel, "algorithmic_bytes": bytes_}
    d.update(extra)
    return d


def _edges_of_levels(levels_dev, deg_dev, directed=False):
    """Traversed edges per row of a (k, n) device level array: arcs leaving
    reached vertices, halved on an undirected graph."""
    arcs = ((levels_dev >= 0).to(deg_dev.dtype) * deg_dev[None, :]).sum(dim=1)
    return arcs if directed else arcs // 2


# ------------------------------------------------------------ per config
def config_c1(ctx):
    """C1: RMAT scale 16, 64 sources, no reordering; the plain method (the
    paper's rule, b1 MMA) is the configuration's figure; the tuned arm too."""
    f, runs = run_single_source(ctx, ["rmat16"], steps=min(ctx.args.steps, 5), warmup=3, tune=True)
    for r in runs:
        r.close()
    rf = f["roofline"]
    rf["note"] = "the graph (10 MB of BVSS) is L2-resident, so the HBM fraction is not meaningful"
    return {"what": "single-source BFS, RMAT scale 16 (65,536 vertices), 64 seeded sources, no reordering",
            "value": f["plain"]["value"], "unit": "GTEPS", "arm": "plain (the paper's rule, b1 MMA, default launch)",
            "tuned": f["value"], "roofline": rf, "levels_bit_exact": f["levels_bit_exact"],
            "sources": f["sources"], "e2e": f["e2e"], "graph": f["graphs"]["rmat16"],
            "gpu_launches": min(ctx.args.steps, 5) * f["sources"]}


def config_c3(ctx):
    """C3: multi-source BFS on RMAT 22 (kappa 64 / 256 / 1024 over the first
    64 / 256 / 1024 of one seeded source draw), the same 1024 sources as
    plain and learned single-source BFSs, and the 10,000-graph BA batch."""
    import oracle
    torch, blest, dev, stream = ctx.torch, ctx.blest, ctx.dev, ctx.stream
    t0 = time.time()
    g = gg.rmat(22, 16, seed=3)
    gen_s = time.time() - t0
    srcs = gg.sources(g, 1024, 22)
    deg = torch.from_numpy(np.diff(g.row_ptr)).to(dev)
    h = blest.build(g.n, g.row_ptr, g.col)
    h.set_stream(stream.cuda_stream, True)
    info = h.info()
    reps = 3

    def time_msbfs(sd, out):
        for _ in range(2):
            h.msbfs(sd, out)
        h.sync()
        a, b = ctx.events()
        a.record(stream)
        for _ in range(reps):
            h.msbfs(sd, out)
        b.record(stream)
        torch.cuda.synchronize()
        h.sync()
        return a.elapsed_time(b) / reps

    outs, per_k, tc_exact = {}, {}, {}
    for k in (64, 256, 1024):
        sd = torch.from_numpy(srcs[:k]).to(dev)
        out = torch.empty((k, g.n), dtype=torch.int32, device=dev)
        # the tcgen05 stage 1 first (its levels kept for the check), then CUDA cores
        h.set_msbfs_engine(True)
        ms_tc = time_msbfs(sd, out)
        st_tc = h.msbfs_stats()
        tc_out = out[:64].clone()
        h.set_msbfs_engine(False)
        ms = time_msbfs(sd, out)
        st = h.msbfs_stats()
        tc_exact[k] = bool(torch.equal(tc_out, out[:64]))
        del tc_out
        edges = torch.cat([_edges_of_levels(out[i:i + 64], deg) for i in range(0, k, 64)]).cpu().numpy()
        nb = msbfs_algorithmic_bytes(st, g.n, info["tau"], 8, levels_out=True)
        per_k[k] = {"ms": ms, "gteps": float(edges.sum()) / (ms * 1e-3) / 1e9, "counters": st,
                    "roofline": _roof(ctx, nb, ms * 1e-3, f"k_msbfs<{k // 32}>"),
                    "tcgen05": {"ms": ms_tc, "gteps": float(edges.sum()) / (ms_tc * 1e-3) / 1e9,
                                "roofline": _roof(ctx, msbfs_algorithmic_bytes(st_tc, g.n, info["tau"], 8), ms_tc * 1e-3,
                                                  f"k_msbfs_tc<{k // 32}>"),
                                "first_64_lanes_equal_cuda_core": tc_exact[k]},
                    "engine": "cuda cores" if ms <= ms_tc else "tcgen05"}
        outs[k] = out
    # levels: every lane of every batch against the oracle (chunks of 64 sources)
    exact = {64: 0, 256: 0, 1024: 0}
    for i in range(0, 1024, 64):
        ref = oracle.bfs_many(g, srcs[i:i + 64])
        for k in (64, 256, 1024):
            if i < k:
                got = outs[k][i:i + 64].cpu().numpy()
                exact[k] += int(sum(np.array_equal(got[j], ref[j]) for j in range(64)))
    edges1024 = torch.cat([_edges_of_levels(outs[1024][i:i + 64], deg) for i in range(0, 1024, 64)]).cpu().numpy()
    for k in (64, 256, 1024):
        per_k[k]["levels_bit_exact"] = exact[k]
        per_k[k]["sources"] = k
    del outs
    # the same 1024 sources as single-source BFSs: plain (rule, b1 MMA, default launch) and learned
    ss = {}
    out1 = torch.empty(g.n, dtype=torch.int32, device=dev)
    if ctx.weights is not None:
        h.load_model(ctx.weights)
    for arm, pol, tc, launch in (("plain", blest.POLICY_HEURISTIC, True, (512, 2)),
                                 ("learned", blest.POLICY_LEARNED if ctx.weights is not None
                                  else blest.POLICY_HEURISTIC, False, (1024, 2))):
        h.set_policy(pol)
        h.set_engine(tc)
        h.set_launch(*launch)
        for s_ in srcs[:8]:
            h.bfs(int(s_), out1)
        h.sync()
        evs = [ctx.events() for _ in srcs]
        for (a, b), s_ in zip(evs, srcs):
            a.record(stream)
            h.bfs(int(s_), out1)
            b.record(stream)
        torch.cuda.synchronize()
        h.sync()
        ms = np.array([a.elapsed_time(b) for a, b in evs])
        rates = edges1024 / (ms * 1e-3) / 1e9
        ss[arm] = {"gteps_harmonic": harmonic(rates), "gteps_aggregate": float(edges1024.sum() / (ms.sum() * 1e-3) / 1e9),
                   "ms_total": float(ms.sum())}
    msa = per_k[1024]["gteps"]
    lbp = {"graph": "RMAT scale 22, edge factor 16", "sources": 1024,
           "batched_gteps": msa, "plain_single_source_gteps": ss["plain"]["gteps_aggregate"],
           "learned_single_source_gteps": ss["learned"]["gteps_aggregate"],
           "batched_over_plain": msa / ss["plain"]["gteps_aggregate"],
           "learned_over_plain": ss["learned"]["gteps_aggregate"] / ss["plain"]["gteps_aggregate"],
           "what": "aggregate GTEPS (sum of traversed edges / total device time) of the 1024 sources: multi-source "
                   "BFS with 1024 lanes against one single-source BFS per source under the paper's rule (b1 MMA, "
                   "default launch) and under the learned policy; levels of every lane checked against the oracle"}
    h.close()
    del g
    # the batch of 10,000 Barabasi-Albert graphs, one launch, every graph checked
    t0 = time.time()
    bt = gg.ba_batch(10000, 1000, 100000, 4, seed=3)
    gen_b = time.time() - t0
    bsrc = np.zeros(bt.g, np.int32)
    hb = blest.build_many(bt)
    hb.set_stream(stream.cuda_stream, True)
    tot = int(bt.vtx_off[-1])
    outb = torch.empty(tot, dtype=torch.int32, device=dev)
    for _ in range(3):
        hb.bfs_many(bsrc, outb)
    hb.sync()
    a, b = ctx.events()
    a.record(stream)
    for _ in range(reps):
        hb.bfs_many(bsrc, outb)
    b.record(stream)
    torch.cuda.synchronize()
    hb.sync()
    msb = a.elapsed_time(b) / reps
    lv = outb.cpu().numpy()
    degs = np.concatenate([np.diff(bt.row_ptr[bt.vtx_off[i] + i: bt.vtx_off[i + 1] + i + 1]) for i in range(bt.g)])
    arcs = int(degs[lv >= 0].sum())
    from concurrent.futures import ThreadPoolExecutor

    def chk(i):
        gi = bt.graph(i)
        return np.array_equal(lv[bt.vtx_off[i]:bt.vtx_off[i + 1]], oracle.bfs(gi, 0))
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        okb = int(sum(ex.map(chk, range(bt.g))))
    hb.close()
    batch = {"what": "10,000 Barabasi-Albert graphs (n log-uniform in [1e3, 1e5], m = 4), one BFS per graph from "
                     "vertex 0, one persistent launch replayed from a CUDA graph",
             "gteps": arcs / 2 / (msb * 1e-3) / 1e9, "ms": msb, "total_vertices": tot, "total_arcs": arcs,
             "levels_bit_exact": okb, "graphs": bt.g, "gen_s": round(gen_b, 1)}
    return {"what": "multi-source BFS on RMAT scale 22 (edge factor 16), 64 / 256 / 1024 lanes over the first "
                    "64 / 256 / 1024 of one seeded draw of sources; the batched small-graph run",
            "value": msa, "unit": "GTEPS", "per_kappa": per_k, "roofline": per_k[1024]["roofline"],
            "levels_bit_exact": exact[1024], "sources": 1024, "single_source_same_sources": ss,
            "learned_batched_vs_plain": lbp, "bfs_many_ba10k": batch, "gen_s": round(gen_s, 1),
            "gpu_launches": reps * 3 + 2 * 1024 + reps}


def config_c4(ctx):
    """C4: all-source closeness on RMAT 18 (far and reach bit-exact and cc
    within 1e-12 at 1024 seeded targets against the oracle), split by source
    ranges over the ranks when there are several; the 2048^2 grid timed
    over its first 8 batches here (the full run is its own workload)."""
    import oracle
    torch, blest, dev, stream, dist = ctx.torch, ctx.blest, ctx.dev, ctx.stream, ctx.dist
    g = gg.rmat(18, 16, seed=4)
    h = blest.build(g.n, g.row_ptr, g.col)
    h.set_stream(stream.cuda_stream, False)
    far = torch.empty(g.n, dtype=torch.int64, device=dev)
    reach = torch.empty(g.n, dtype=torch.int64, device=dev)
    # the tcgen05 stage 1 timed first, then the CUDA-core one (whose result is checked)
    h.set_msbfs_engine(True)
    h.closeness_range(0, 1024, far, reach)            # warm-up (captures the batch graph)
    torch.cuda.synchronize()
    ms_tc, f_tc, r_tc, _, _ = closeness_split_run(h, g.n, ctx.rank, ctx.world, dist, far, reach, CudaTimer(ctx))
    h.set_msbfs_engine(False)
    h.closeness_range(0, 1024, far, reach)
    torch.cuda.synchronize()
    ms, f_all, r_all, cc, (_, count) = closeness_split_run(h, g.n, ctx.rank, ctx.world, dist, far, reach,
                                                           CudaTimer(ctx))
    st = h.msbfs_stats()
    tc_equal = bool(np.array_equal(f_tc, f_all) and np.array_equal(r_tc, r_all))
    tg = gg.sources(g, 1024, 18)
    fr, rr = oracle.far_reach(g, tg)
    cc_ref = oracle.closeness_from(fr, rr)
    exact = int(np.sum((f_all[tg] == fr) & (r_all[tg] == rr)))
    rel = np.abs(cc[tg] - cc_ref) / np.maximum(np.abs(cc_ref), 1e-300)
    nb = msbfs_algorithmic_bytes(st, g.n, h.info()["tau"], 8, levels_out=False, closeness=True)
    pairs = int(r_all.sum())
    h.close()
    rmat18 = {"what": "all 262,144 sources of RMAT scale 18 (edge factor 16), 256 batches of 1024",
              "seconds": ms * 1e-3, "bfs_per_s": g.n / (ms * 1e-3),
              "gteps_est": pairs * (g.nnz / g.n) / 2 / (ms * 1e-3) / 1e9,
              "targets_checked": len(tg), "far_reach_bit_exact": exact, "cc_max_rel_err": float(rel.max()),
              "roofline": _roof(ctx, nb, ms * 1e-3 / max(1, ctx.world) * ctx.world, "k_msbfs<32>",
                                note="the graph is L2-resident; the HBM fraction is not meaningful"),
              "counters": st, "ranks": ctx.world,
              "tcgen05": {"seconds": ms_tc * 1e-3, "far_reach_equal_cuda_core": tc_equal},
              "engine": "cuda cores" if ms <= ms_tc else "tcgen05"}
    # the grid: 8 of its 4096 batches, as a time estimate
    gq = gg.grid(2048, 2048, 0.05, 0.001, seed=4)
    hq = blest.build(gq.n, gq.row_ptr, gq.col, tau=32)
    hq.set_stream(stream.cuda_stream, False)
    fq = torch.empty(gq.n, dtype=torch.int64, device=dev)
    rq = torch.empty(gq.n, dtype=torch.int64, device=dev)
    hq.closeness_range(0, 1024, fq, rq)
    torch.cuda.synchronize()
    a, b = ctx.events()
    a.record(stream)
    hq.closeness_range(0, 8 * 1024, fq, rq)
    b.record(stream)
    torch.cuda.synchronize()
    msq = a.elapsed_time(b)
    stq = hq.msbfs_stats()
    nbq = msbfs_algorithmic_bytes(stq, gq.n, 32, 8, levels_out=False, closeness=True)
    hq.close()
    grid = {"what": "2048^2 road-like grid (tau 32), sources 0..8191 (8 of 4096 batches)", "ms": msq,
            "full_run_estimate_s": (gq.n / 8192) * msq * 1e-3,
            "roofline": _roof(ctx, nbq, msq * 1e-3, "k_msbfs<32>"), "counters": stq,
            "full_run": _full_grid_record()}
    return {"what": "exact closeness (far bit-exact, cc within 1e-12) by all-source multi-source BFS",
            "value": rmat18["bfs_per_s"], "unit": "BFS/s", "rmat18": rmat18, "grid2048": grid,
            "levels_bit_exact": exact, "sources": len(tg), "roofline": rmat18["roofline"],
            "gpu_launches": (count + 1023) // 1024 + 8}


class CudaTimer:
    """CUDA events on the library's stream around a region (milliseconds)."""

    def __init__(self, ctx):
        self.ctx = ctx

    def start(self):
        self.a, self.b = self.ctx.events()
        self.a.record(self.ctx.stream)

    def stop(self):
        self.b.record(self.ctx.stream)
        self.ctx.torch.cuda.synchronize()
        return self.a.elapsed_time(self.b)


def closeness_split_run(h, n, rank, world, dist, far, reach, timer):
    """All-source closeness split over the ranks: this rank runs the
    multi-source batches of its own source range (between a barrier and the
    timer's stop), then one integer all-reduce of far and reach completes
    the result on every rank.  Returns (max-over-ranks ms, far, reach, cc,
    (first, count)) with far, reach, cc as host arrays."""
    import torch
    from paper_2606_05081_gb300 import distributed
    first, count = distributed.source_ranges(n, world)[rank]
    if dist is not None and world > 1:
        dist.barrier()
    timer.start()
    h.closeness_range(first, count, far, reach)
    ms = timer.stop()
    if dist is not None and world > 1:
        tt = torch.tensor([ms], dtype=torch.float64, device=distributed.reduce_device(dist))
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    f_all, r_all, cc = distributed.closeness_allreduce(lambda f0, c0: (far, reach), n, rank, world,
                                                       dist if world > 1 else None)
    return ms, f_all, r_all, cc, (first, count)


def _full_grid_record():
    """The committed record of the full 2048^2 grid closeness run (its own
    workload, too long for this run), when one exists."""
    p = os.path.join(ROOT, "profiles", "closeness_grid2048_full.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except ValueError:
        return None
    d["kernel_sources_unchanged"] = d.get("kernel_sha") == kernel_sha(MS_KERNEL_SOURCES)
    return d


def config_c5(ctx):
    """C5: the learned policy against the paper's rule on graph families it
    was not trained on -- levels of all 64 sources bit-exact, GTEPS of both
    policies, and time regret against the per-level optimum."""
    import oracle
    from paper_2606_05081_gb300 import switch
    torch, blest, dev, stream = ctx.torch, ctx.blest, ctx.dev, ctx.stream
    w = ctx.weights
    if w is None:
        return {"value": None, "unavailable": "no trained weights"}
    fams = [("rmat25", lambda: gg.rmat(25, 16, seed=25), "RMAT scale 25, edge factor 16"),
            ("ba16m_m8", lambda: gg.ba(1 << 24, 8, seed=26), "Barabasi-Albert, 2^24 vertices, m = 8"),
            ("rgg16m", lambda: gg.rgg(1 << 24, 10.0, seed=27), "random geometric, 2^24 points, average degree 10")]
    per, regs, ex_tot, n_tot, hrates = {}, [], 0, 0, []
    launches = 0
    for name, mk, desc in fams:
        t0 = time.time()
        g = mk()
        gen_s = time.time() - t0
        srcs = gg.sources(g, NUM_SOURCES, 5)
        h = blest.build(g.n, g.row_ptr, g.col)
        h.set_stream(stream.cuda_stream, True)
        h.load_model(w)
        ev = switch.evaluate(h, srcs[:8], w, reps=2)
        deg = torch.from_numpy(np.diff(g.row_ptr)).to(dev)
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
        res = {}
        for pol, tc in (("learned", False), ("heuristic", True)):
            h.set_engine(tc)
            h.set_policy(blest.POLICY_LEARNED if pol == "learned" else blest.POLICY_HEURISTIC)
            for s_ in srcs[:4]:
                h.bfs(int(s_), out)
            h.sync()
            ms, edges = [], []
            for s_ in srcs:
                a, b = ctx.events()
                a.record(stream)
                h.bfs(int(s_), out)
                b.record(stream)
                torch.cuda.synchronize()
                h.sync()
                ms.append(a.elapsed_time(b))
                edges.append(int(_edges_of_levels(out[None, :], deg)[0].item()))
                launches += 1
            ms, edges = np.array(ms), np.array(edges, np.float64)
            rates = edges / (ms * 1e-3) / 1e9
            res[pol] = {"gteps_harmonic": harmonic(rates), "gteps_aggregate": float(edges.sum() / (ms.sum() * 1e-3) / 1e9),
                        "small_component_sources": int(np.sum(edges < 1000))}
        h.set_engine(False)
        h.set_policy(blest.POLICY_LEARNED)
        h.set_stream(None, False)
        exact = levels_exact_single(g, srcs, h, torch, dev)
        ex_tot += exact
        n_tot += len(srcs)
        hrates.append(res["learned"]["gteps_harmonic"])
        per[name] = {"graph": desc, "n": g.n, "nnz": g.nnz, "gen_s": round(gen_s, 1),
                     "levels_bit_exact": exact, "sources": len(srcs),
                     "regret_learned": ev["regret_learned"], "regret_heuristic_tc": ev["regret_heuristic_tc"],
                     "regret_heuristic_cc": ev["regret_heuristic_cc"], "ms_learned": ev["ms_learned"],
                     "ms_heuristic_tc": ev["ms_heuristic_tc"], "ms_optimal": ev["ms_optimal"],
                     "gteps_learned": res["learned"], "gteps_heuristic_tc": res["heuristic"]}
        regs.append(ev["regret_learned"])
        h.close()
        del g
    return {"what": "learned level-mode policy vs the paper's rule (b1 MMA) on held-out families; regret = time "
                    "over the per-level optimum on 8 sources, GTEPS on all 64",
            "value": float(np.mean(regs)), "unit": "mean time regret of the learned policy",
            "higher_is_better": False, "per_family": per, "levels_bit_exact": ex_tot, "sources": n_tot,
            "gpu_launches": launches}


PER_CONFIG = {"C1": config_c1, "C3": config_c3, "C4": config_c4, "C5": config_c5}


def run_extra(args, ctx):
    """One row of the path on its own JSON line (multi-source BFS, closeness,
    the batched small graphs, the held-out policy evaluation)."""
    line = {"n_gpus": ctx.world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic"}
    if args.workload == "msbfs_rmat22":
        c = config_c3(ctx)
        line.update({"metric": "GTEPS (aggregate over sources), multi-source BFS", "value": c["value"],
                     "unit": "GTEPS", "ms_per_step": c["per_kappa"][1024]["ms"],
                     "config": {"workload": args.workload, "graph": "RMAT scale 22, edge factor 16",
                                "kappa": [64, 256, 1024], "levels": "int32, source-major"},
                     **{k: c[k] for k in ("per_kappa", "roofline", "levels_bit_exact", "sources",
                                          "learned_batched_vs_plain", "bfs_many_ba10k", "gpu_launches")}})
    elif args.workload == "bfs_many_ba10k":
        c = config_c3(ctx)["bfs_many_ba10k"]
        line.update({"metric": "GTEPS (aggregate), batched BFS over 10,000 BA graphs", "value": c["gteps"],
                     "unit": "GTEPS", "ms_per_step": c["ms"], "config": {"workload": args.workload},
                     "batch": c, "gpu_launches": 3})
    elif args.workload == "closeness_rmat18" or args.workload == "closeness_grid2048_part":
        c = config_c4(ctx)
        line.update({"metric": "BFS per second, all-source closeness", "value": c["value"], "unit": "BFS/s",
                     "config": {"workload": args.workload}, "rmat18": c["rmat18"], "grid2048": c["grid2048"],
                     "gpu_launches": c["gpu_launches"]})
    elif args.workload == "closeness_grid2048":
        line.update(run_grid_closeness_full(args, ctx))
    elif args.workload == "msbfs_one":
        line.update(run_msbfs_one(args, ctx))
    elif args.workload == "ablation":
        line.update(run_ablation(args, ctx))
    elif args.workload == "order_study":
        line.update(run_order_study(args, ctx))
    elif args.workload == "switch_heldout":
        c = config_c5(ctx)
        line.update({"metric": "switching regret of the learned policy (held-out families), mean",
                     "config": {"workload": args.workload}, **c})
    if ctx.rank == 0:
        print(json.dumps(line), flush=True)


def _time_sources(ctx, h, srcs, out, warm=3):
    """Device time (ms) of one BFS from each source, CUDA events on the
    library's stream."""
    torch, stream = ctx.torch, ctx.stream
    for s_ in srcs[:warm]:
        h.bfs(int(s_), out)
    h.sync()
    evs = [ctx.events() for _ in srcs]
    for (a, b), s_ in zip(evs, srcs):
        a.record(stream)
        h.bfs(int(s_), out)
        b.record(stream)
    torch.cuda.synchronize()
    h.sync()
    return np.array([a.elapsed_time(b) for a, b in evs])


def run_msbfs_one(args, ctx):
    """One multi-source configuration (RMAT --scale, --kappa sources, stage 1
    on CUDA cores or tcgen05): W warm-up and K timed launches, the levels of
    the first lanes checked against the oracle; small enough to profile."""
    import oracle
    torch, blest, dev, stream = ctx.torch, ctx.blest, ctx.dev, ctx.stream
    g = gg.rmat(args.scale, 16, seed=3)
    srcs = gg.sources(g, args.kappa, 22)
    h = blest.build(g.n, g.row_ptr, g.col)
    h.set_stream(stream.cuda_stream, True)
    h.set_msbfs_engine(args.engine == "tc")
    h.set_msbfs_direction(args.direction)
    h.set_msbfs_output(bool(args.staged))
    sd = torch.from_numpy(srcs).to(dev)
    out = torch.empty((len(srcs), g.n), dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        h.msbfs(sd, out)
    h.sync()
    a, b = ctx.events()
    a.record(stream)
    for _ in range(args.steps):
        h.msbfs(sd, out)
    b.record(stream)
    torch.cuda.synchronize()
    h.sync()
    ms = a.elapsed_time(b) / args.steps
    st = h.msbfs_stats()
    chk = min(16, len(srcs))
    ok = int(np.array_equal(out[:chk].cpu().numpy(), oracle.bfs_many(g, srcs[:chk])))
    deg = torch.from_numpy(np.diff(g.row_ptr)).to(dev)
    edges = float(torch.cat([_edges_of_levels(out[i:i + 64], deg) for i in range(0, len(srcs), 64)]).sum().item())
    nb = msbfs_algorithmic_bytes(st, g.n, 128, 8, levels_out=True)
    h.close()
    return {"metric": "GTEPS (aggregate), one multi-source configuration", "value": edges / (ms * 1e-3) / 1e9,
            "unit": "GTEPS", "ms_per_step": ms,
            "config": {"workload": "msbfs_one", "graph": f"RMAT scale {args.scale}, edge factor 16",
                       "kappa": len(srcs), "engine": args.engine, "direction": args.direction,
                       "staged_output": args.staged},
            "counters": st, "first_lanes_exact": bool(ok),
            "roofline": _roof(ctx, nb, ms * 1e-3, ("k_msbfs_tc" if args.engine == "tc" else "k_msbfs")),
            "gpu_launches": args.steps}


def run_ablation(args, ctx):
    """The ablation ladders of §7.1 on GB300.

    Single-source (64 sources each on RMAT 24 and the 4096^2 grid), each rung
    adding one optimisation: (A) BVSS + kernel fusion, eager updates, b1 MMA
    with one slice per fragment row (16 MMAs per VSS), no reordering; (AB) +
    the optimal layout of Fig. 3 (2 MMAs per VSS); (ABC) + reordering
    (JaccardWithWindows / RCM); (ABCD) + lazy updates by the U_div rule;
    (Full) + Eq. 5 switching (the paper's method); then this build's steps:
    CUDA-core hit test; learned level policy.  Multi-source (256 sources on
    RMAT 22 and the 2048^2 grid): (Naive) 256 single-source BFSs of the full
    method; (A) Algorithm 5 without getVI reindexing or activeSets /
    dirtySets tracking; (AB) without tracking; (Full) Algorithm 5 (push);
    (Full, tcgen05) its stage 1 on the tensor cores; then this build's
    direction-optimizing stage 1 (pull on dense levels, pull always).  Levels of a sample of sources
    per rung are checked against the oracle."""
    import oracle
    torch, blest, dev, stream = ctx.torch, ctx.blest, ctx.dev, ctx.stream
    out_ss = {}
    specs = [("rmat24", lambda: gg.rmat(24, 16, seed=2), dict(reorder=REORDER_JACCARD, jaccard_window=65536)),
             ("grid4096", lambda: gg.grid(4096, 4096, 0.05, 0.001, seed=2), dict(reorder=REORDER_RCM))]
    for name, mk, ropt in specs:
        g = mk()
        srcs = gg.sources(g, args.sources, 7)
        chk = srcs[:4]
        ref = oracle.bfs_many(g, chk)
        deg = np.diff(g.row_ptr)
        h0 = blest.build(g.n, g.row_ptr, g.col)
        h1 = blest.build(g.n, g.row_ptr, g.col, **ropt)
        for h in (h0, h1):
            h.set_stream(stream.cuda_stream, True)
            if ctx.weights is not None:
                h.load_model(ctx.weights)
        built_switch = h1.info()["switching"]
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
        rungs = [("A", h0, 2, blest.POLICY_FIXED, 1, None),
                 ("AB", h0, 1, blest.POLICY_FIXED, 1, None),
                 ("ABC", h1, 1, blest.POLICY_FIXED, 1, None),
                 ("ABCD", h1, 1, blest.POLICY_HEURISTIC, 0, 0),
                 ("Full", h1, 1, blest.POLICY_HEURISTIC, 0, built_switch),
                 ("Full, CUDA-core hit test", h1, 0, blest.POLICY_HEURISTIC, 0, built_switch)]
        if ctx.weights is not None:
            rungs.append(("Full, learned level policy", h1, 0, blest.POLICY_LEARNED, 0, built_switch))
        res = {}
        edges = None
        for rung, h, eng, pol, mode, sw in rungs:
            h.set_engine(eng)
            h.set_policy(pol, mode)
            if sw is not None:
                h.set_switching(sw)
            h.set_launch(512, 2)
            ms = _time_sources(ctx, h, srcs, out)
            ok = 0
            for j, s_ in enumerate(chk):
                h.bfs(int(s_), out)
                h.sync()
                ok += int(np.array_equal(out.cpu().numpy(), ref[j]))
            if edges is None:
                edges = []
                for s_ in srcs:
                    h.bfs(int(s_), out)
                    h.sync()
                    lv = out.cpu().numpy()
                    edges.append(int(deg[lv >= 0].sum()) // 2)
                edges = np.array(edges, np.float64)
            res[rung] = {"ms_mean": float(ms.mean()), "gteps_harmonic": harmonic(edges / (ms * 1e-3) / 1e9),
                         "levels_bit_exact_checked": ok, "checked": len(chk)}
        base = res["A"]["ms_mean"]
        for v in res.values():
            v["speedup_vs_A"] = base / v["ms_mean"]
        out_ss[name] = {"n": g.n, "nnz": g.nnz, "udiv_reordered": h1.info()["update_divergence"],
                        "switching_built": built_switch, "rungs": res}
        h0.close()
        h1.close()
        del g
    # multi-source ladder
    out_ms = {}
    for name, mk, tau in [("rmat22", lambda: gg.rmat(22, 16, seed=3), 128),
                          ("grid2048", lambda: gg.grid(2048, 2048, 0.05, 0.001, seed=4), 32)]:
        g = mk()
        srcs = gg.sources(g, 256, 22)
        ref = oracle.bfs_many(g, srcs)
        h = blest.build(g.n, g.row_ptr, g.col, tau=tau)
        h.set_stream(stream.cuda_stream, True)
        sd = torch.from_numpy(srcs).to(dev)
        out = torch.empty((len(srcs), g.n), dtype=torch.int32, device=dev)
        res = {}
        # Naive: one single-source BFS per source, the paper's full method
        out1 = torch.empty(g.n, dtype=torch.int32, device=dev)
        h.set_engine(1 if tau == 128 else 0)
        h.set_policy(blest.POLICY_HEURISTIC)
        ms = _time_sources(ctx, h, srcs, out1)
        res["Naive"] = {"seconds": float(ms.sum()) * 1e-3}
        # (rung, (reindex, tracking), tcgen05 stage 1, direction, staged level output)
        variants = [("A", (0, 0), 0, 0, 0), ("AB", (1, 0), 0, 0, 0), ("Full", (1, 1), 0, 0, 0),
                    ("Full, staged level output", (1, 1), 0, 0, 1)]
        if tau == 128:
            variants.append(("Full, staged, tcgen05 stage 1", (1, 1), 1, 0, 1))
        variants += [("Full, staged, pull on dense levels", (1, 1), 0, 1, 1),
                     ("Full, staged, pull on every level", (1, 1), 0, 2, 1)]
        for rung, (ri, tr), eng, direction, staged in variants:
            h.set_msbfs_engine(False)
            h.set_msbfs_variant(ri, tr)
            h.set_msbfs_engine(bool(eng))
            h.set_msbfs_direction(direction)
            h.set_msbfs_output(bool(staged))
            h.msbfs(sd, out)
            h.sync()
            a, b = ctx.events()
            a.record(stream)
            h.msbfs(sd, out)
            b.record(stream)
            torch.cuda.synchronize()
            h.sync()
            got = out.cpu().numpy()
            res[rung] = {"seconds": a.elapsed_time(b) * 1e-3,
                         "levels_bit_exact": int(sum(np.array_equal(got[j], ref[j]) for j in range(len(srcs)))),
                         "counters": h.msbfs_stats()}
        for v in res.values():
            v["speedup_vs_naive"] = res["Naive"]["seconds"] / v["seconds"]
        out_ms[name] = {"n": g.n, "nnz": g.nnz, "tau": tau, "sources": len(srcs), "rungs": res}
        h.close()
        del g
    return {"metric": "ablation ladders (ms per single-source BFS, seconds per 256-source batch)", "value": None,
            "unit": "see rungs", "config": {"workload": "ablation", "sources": args.sources},
            "single_source": out_ss, "multi_source": out_ms, "gpu_launches": None}


def run_order_study(args, ctx):
    """The ordering experiments of §7.1 on RMAT 24: the JaccardWithWindows
    window W from 2^3 to 2^18 (BVSS size and BFS time), RCM, the scale-free
    test's choice, no reordering of the generator's scrambled labels (a
    random order) and of its unscrambled labels (the natural RMAT order:
    hubs first).  Per order: VSS and slice counts, U_div, and the mean
    device time per BFS of the (AB) rung (eager updates, Fig. 3 b1 MMA), the
    paper's rule (Full) and the learned policy, 8 sources each."""
    import oracle
    torch, blest, dev, stream = ctx.torch, ctx.blest, ctx.dev, ctx.stream
    out = torch.empty(1 << 24, dtype=torch.int32, device=dev)
    res = {}

    def measure(label, g, srcs, opt):
        t0 = time.time()
        h = blest.build(g.n, g.row_ptr, g.col, **opt)
        inf = h.info()
        row = {"build_s": round(time.time() - t0, 2), "num_vss": inf["num_vss"], "num_slices": inf["num_slices"],
               "udiv": inf["update_divergence"], "lazy": inf["lazy"], "reorder": inf["reorder"]}
        h.set_stream(stream.cuda_stream, True)
        if ctx.weights is not None:
            h.load_model(ctx.weights)
        for key, pol, mode, eng in (("AB_ms", blest.POLICY_FIXED, 1, 1), ("rule_ms", blest.POLICY_HEURISTIC, 0, 1),
                                    ("learned_ms", blest.POLICY_LEARNED, 0, 0)):
            if pol == blest.POLICY_LEARNED and ctx.weights is None:
                continue
            h.set_engine(eng)
            h.set_policy(pol, mode)
            row[key] = float(_time_sources(ctx, h, srcs, out[:g.n]).mean())
        h.set_stream(None, False)
        row["levels_exact_source0"] = bool(np.array_equal(h.bfs(int(srcs[0])), oracle.bfs(g, int(srcs[0]))))
        res[label] = row
        h.close()

    g = gg.rmat(24, 16, seed=2)
    srcs = gg.sources(g, 8, 7)
    for label, opt in [("scrambled (random order)", dict(reorder=0)), ("rcm", dict(reorder=REORDER_RCM)),
                       ("auto", dict(reorder=3, jaccard_window=65536))] + \
                      [(f"jaccard W=2^{e}", dict(reorder=REORDER_JACCARD, jaccard_window=1 << e))
                       for e in range(3, 19)]:
        measure(label, g, srcs, opt)
    del g
    g = gg.rmat(24, 16, seed=2, scramble=False)
    measure("natural (unscrambled RMAT labels)", g, gg.sources(g, 8, 7), dict(reorder=0))
    return {"metric": "ms per single-source BFS under each vertex order (RMAT 24)", "value": None, "unit": "ms",
            "config": {"workload": "order_study", "graph": "RMAT scale 24, edge factor 16", "sources": 8},
            "orders": res, "gpu_launches": None}


def run_grid_closeness_full(args, ctx):
    """Config 4's grid: exact closeness over all 4,194,304 sources of the
    2048^2 road-like grid (4096 batches of 1024 lanes), split over the ranks
    by source ranges; far and reach checked bit-exact and cc within 1e-12 at
    256 seeded targets against the oracle."""
    import oracle
    torch, blest, dev, stream, dist = ctx.torch, ctx.blest, ctx.dev, ctx.stream, ctx.dist
    g = gg.grid(2048, 2048, 0.05, 0.001, seed=4)
    h = blest.build(g.n, g.row_ptr, g.col, tau=32)
    h.set_stream(stream.cuda_stream, False)
    far = torch.empty(g.n, dtype=torch.int64, device=dev)
    reach = torch.empty(g.n, dtype=torch.int64, device=dev)
    h.closeness_range(0, 1024, far, reach)
    torch.cuda.synchronize()
    with ClockSampler(ctx.local) as clk:
        ms, f_all, r_all, cc, (_, count) = closeness_split_run(h, g.n, ctx.rank, ctx.world, dist, far, reach,
                                                               CudaTimer(ctx))
    st = h.msbfs_stats()
    tg = gg.sources(g, 256, 2048)
    fr, rr = oracle.far_reach(g, tg)
    cc_ref = oracle.closeness_from(fr, rr)
    exact = int(np.sum((f_all[tg] == fr) & (r_all[tg] == rr)))
    rel = np.abs(cc[tg] - cc_ref) / np.maximum(np.abs(cc_ref), 1e-300)
    nb = msbfs_algorithmic_bytes(st, g.n, 32, 8, levels_out=False, closeness=True)
    h.close()
    return {"metric": "seconds, exact all-source closeness of the 2048^2 road-like grid", "value": ms * 1e-3,
            "unit": "s", "higher_is_better": False, "ms_per_step": ms,
            "config": {"workload": "closeness_grid2048", "graph": "2048x2048 4-neighbour grid, 5% edges deleted, "
                       "0.1% random shortcuts, no reordering, tau 32", "n": g.n, "nnz": g.nnz,
                       "batches": (g.n + 1023) // 1024},
            "bfs_per_s": g.n / (ms * 1e-3), "targets_checked": len(tg), "far_reach_bit_exact": exact,
            "cc_max_rel_err": float(rel.max()), "counters": st,
            "roofline": _roof(ctx, nb, ms * 1e-3, "k_msbfs<32>"), "clocks": clk.summary(),
            "kernel_sha": kernel_sha(MS_KERNEL_SOURCES), "gpu_launches": (count + 1023) // 1024}


if __name__ == "__main__":
    main()
