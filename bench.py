"""Benchmark: single-source BFS throughput (GTEPS, harmonic mean over seeded
sources) of the BVSS path on one GB300, with its HBM roofline fraction.

Default workload (the single-source configuration): 64 seeded sources on
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
    "sssp_pair": ["rmat24_jaccard", "grid4096_rcm"],
    "rmat24": ["rmat24"],
    "rmat22": ["rmat22"],
    "rmat16": ["rmat16"],
    "grid4096_rcm": ["grid4096_rcm"],
    "rmat24_jaccard": ["rmat24_jaccard"],
}
DEFAULT_WORKLOAD = "sssp_pair"
# the other rows of the path, each with its own JSON line
EXTRA_WORKLOADS = ["msbfs_rmat22", "closeness_rmat18", "closeness_grid2048_part", "bfs_many_ba10k",
                   "switch_heldout"]
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


def kernel_sha() -> str:
    import hashlib
    hsh = hashlib.sha256()
    for f in KERNEL_SOURCES:
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
    if args.workload in EXTRA_WORKLOADS:
        run_extra(args, rank, world, local)
        if dist:
            dist.destroy_process_group()
        return

    import torch
    import paper_2606_05081_gb300 as blest
    from paper_2606_05081_gb300 import autotune, switch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)

    runs = [GraphRun(nm, args, rank, dev, torch, blest, stream) for nm in WORKLOADS[args.workload]]
    weights = switch.load_weights()
    tuned_policy = blest.POLICY_LEARNED if weights is not None else blest.POLICY_HEURISTIC
    tune_info = {}
    for r in runs:
        if weights is not None:
            r.h.load_model(weights)
        if not args.no_tune:
            r.h_tuned, tune_info[r.name] = autotune.autotune_layout(
                lambda sg, ta, r=r: r.build_layout(blest, sg, ta, weights, tuned_policy), r.tune_srcs, reps=2,
                stream=stream)
        elif args.layout:
            sg, ta = (int(x) for x in args.layout.split(","))
            r.h_tuned = r.build_layout(blest, sg, ta, weights, tuned_policy)
        if args.no_tune and args.launch:
            bt, bb = (int(x) for x in args.launch.split(","))
            tune_info[r.name] = {"block_threads": bt, "vss_batch": bb, "engine_tc": 0, "fixed": True}
        r.h_tuned.set_stream(stream.cuda_stream, True)
        ti = tune_info.get(r.name, {})
        r.tuned = (int(ti.get("block_threads", 512)), int(ti.get("vss_batch", 2)), bool(ti.get("engine_tc", 0)))
        if args.levels and rank == 0:
            r.h_tuned.set_policy(tuned_policy)
            for rec in r.logs(r.h_tuned)[0]:
                print(r.name, "level", json.dumps(rec), file=sys.stderr)

    arms = {"plain": (blest.POLICY_HEURISTIC, "default", True), "tuned": (tuned_policy, "tuned", None)}
    if args.ablation:
        arms = {"plain": arms["plain"],
                "rule_cc": (blest.POLICY_HEURISTIC, "default", False),
                "rule_cc_tuned": (blest.POLICY_HEURISTIC, "tuned", False),
                "tuned": arms["tuned"]}

    def set_arm(r, arm):
        """The arm's handle, configured: plain = default layout and launch,
        the paper's rule with the b1 MMA hit test; tuned = the autotuner's
        layout and launch under the learned policy."""
        pol, launch, tc = arms[arm]
        h = r.h if arm == "plain" else r.h_tuned
        if launch == "default":
            h.set_launch(512, 2)
        else:
            h.set_launch(r.tuned[0], r.tuned[1])
        h.set_engine(r.tuned[2] if tc is None else tc)
        h.set_policy(pol)
        return h

    results = {}
    with ClockSampler(local) as clk:
        for arm in arms:
            for r in runs:
                h = set_arm(r, arm)
                for _ in range(args.warmup):
                    r.step(h, False)
                h.sync()
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            psm = {r.name: np.zeros((args.steps, len(r.srcs))) for r in runs}
            t0e.record(stream)
            nvtx_range("timed_" + arm)
            for k in range(args.steps):
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
    hbm, peak_kind = peaks()
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
                                  "algorithmic_bytes_per_launch": gb / len(r.srcs)}
    achieved = alg_b / dev_s / 1e9

    # end to end through the C ABI with host buffers, headline arm
    e2e_rates, d2h = [], 0
    for r in runs:
        h = set_arm(r, "tuned")
        h.set_stream(None, False)
        host = torch.empty(r.g.n, dtype=torch.int32).pin_memory().numpy()
        for s, e in zip(r.srcs, r.edges):
            t0 = time.perf_counter()
            h.bfs(int(s), host)
            e2e_rates.append(e / (time.perf_counter() - t0) / 1e9)
        d2h += 4 * r.g.n * len(r.srcs)
    e2e = harmonic(e2e_rates)

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
            "levels_source0_tuned": [[x["mode"], x["queue"], round(x["t_ns"] / 1e3, 1)]
                                     for x in results["tuned"][2][r.name][0]][:40]}
    line = {
        "metric": METRIC, "value": value, "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": results["tuned"][1] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": args.workload, "sources_per_graph": args.sources,
                   "policy": "learned+autotuned" if weights is not None else "heuristic+autotuned",
                   "l2": "inputs larger than L2 (BVSS arrays), no flush", "parallelism": f"replicas{world}",
                   "graphs": graphs_cfg},
        "plain": {"value": plain_value, "ms_per_step": results["plain"][1] / args.steps,
                  "what": "hand-set rule (U_div lazy/eager, Eq. 5 switch), b1 MMA hit test, default launch"},
        "speedup_vs_plain": value / plain_value,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                     "traffic": measured_traffic([(r.name, r.h_tuned.info()["sigma"], r.h_tuned.info()["tau"])
                                                  for r in runs]), "peak_kind": peak_kind,
                     "kernel": "k_bfs (persistent, all levels)",
                     "algorithmic_bytes_per_launch": alg_b / sum(len(r.srcs) for r in runs),
                     "kernel_sha": kernel_sha(), "per_graph": per_graph_roof},
        "e2e": {"value": e2e, "unit": "GTEPS", "h2d_bytes_per_step": 4 * sum(len(r.srcs) for r in runs),
                "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps * sum(len(r.srcs) for r in runs),   # one k_bfs per BFS of the tuned arm
        "clocks": clk.summary(),
        "autotune": {k: {kk: vv for kk, vv in v.items() if kk != "tried"} for k, v in tune_info.items()},
    }
    if args.ablation:
        what = {"plain": "the paper's rule, b1 MMA hit test, sigma 8 / tau 128, 512-thread CTAs",
                "rule_cc": "the paper's rule, CUDA-core hit test, sigma 8 / tau 128, 512-thread CTAs",
                "rule_cc_tuned": "the paper's rule, CUDA-core hit test, autotuned layout and launch",
                "tuned": "learned per-level policy, autotuned layout and launch"}
        line["ablation"] = {}
        for arm in arms:
            v, per = gteps_of(results[arm][0])
            line["ablation"][arm] = {"value": v, "per_graph": per, "what": what[arm]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rates = []
        for r in runs:
            rates += cpu_sample(r.g, r.srcs, 12.0 / len(runs))
        line["cpu_baseline"] = {"value": harmonic(rates), "unit": "GTEPS", "cores": 1, "kind": "oracle",
                                "sample": f"{len(rates)} of the workload's sources (all graphs), one serial "
                                          "FIFO BFS each on one host core, about 12 s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    for r in runs:
        r.close()
    if dist:
        dist.destroy_process_group()


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_extra(args, rank, world, local):
    """Multi-source BFS (§6.1), closeness (§6.2) and batched small graphs:
    device time with CUDA events on the library's stream, inputs resident."""
    import torch
    import paper_2606_05081_gb300 as blest
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    hbm, peak_kind = peaks()
    line = {"n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic"}
    if args.workload == "msbfs_rmat22":
        g = gg.rmat(22, 16, seed=3)
        h = blest.build(g.n, g.row_ptr, g.col, tau=args.tau)
        h.set_stream(stream.cuda_stream, True)
        deg = torch.from_numpy(np.diff(g.row_ptr)).to(dev)
        res = {}
        for k in (64, 256, 1024):
            srcs = gg.sources(g, k, 22 + k)
            out = torch.empty((k, g.n), dtype=torch.int32, device=dev)
            sd = torch.from_numpy(srcs).to(dev)
            for _ in range(args.warmup):
                h.msbfs(sd, out)
            h.sync()
            a, b = _events(torch)
            a.record(stream)
            for _ in range(args.steps):
                h.msbfs(sd, out)
            b.record(stream)
            torch.cuda.synchronize()
            h.sync()
            ms = a.elapsed_time(b) / args.steps
            reached = out >= 0
            arcs = int((reached.to(torch.int64) * deg[None, :]).sum().item())
            floor = 8.0 * k * g.n      # -1 initialisation and one level write per (source, vertex)
            res[k] = {"ms": ms, "gteps": arcs / 2 / (ms * 1e-3) / 1e9,
                      "level_floor_gbs": floor / (ms * 1e-3) / 1e9}
            del out
        line.update({"metric": "GTEPS (aggregate over sources), multi-source BFS", "value": res[1024]["gteps"],
                     "unit": "GTEPS", "ms_per_step": res[1024]["ms"],
                     "config": {"workload": args.workload, "graph": "RMAT scale 22, edge factor 16", "n": g.n,
                                "nnz": g.nnz, "kappa": [64, 256, 1024], "levels": "int32, source-major"},
                     "per_kappa": res,
                     "roofline": {"bound": "hbm", "achieved": res[1024]["level_floor_gbs"], "peak": hbm,
                                  "unit": "GB/s", "frac": res[1024]["level_floor_gbs"] / hbm, "traffic": None,
                                  "peak_kind": peak_kind,
                                  "bytes": "level-array floor only: 8 B per (source, vertex)"},
                     "gpu_launches": args.steps * 3})
    elif args.workload.startswith("closeness"):
        if args.workload == "closeness_rmat18":
            g = gg.rmat(18, 16, seed=4)
            first, count = 0, g.n
            desc = "RMAT scale 18, edge factor 16, all sources"
        else:
            g = gg.grid(2048, 2048, 0.05, 0.001, seed=4)
            first, count = 0, 8 * 1024
            desc = "2048x2048 road-like grid, sources 0..8191 (8 of the 4096 batches of 1024)"
        h = blest.build(g.n, g.row_ptr, g.col, tau=args.tau)
        h.set_stream(stream.cuda_stream, False)
        far = torch.empty(g.n, dtype=torch.int64, device=dev)
        reach = torch.empty(g.n, dtype=torch.int64, device=dev)
        h.closeness_range(first, min(1024, count), far, reach)
        torch.cuda.synchronize()
        a, b = _events(torch)
        a.record(stream)
        h.closeness_range(first, count, far, reach)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        # traversed edges: each source reaches its component; sum over targets of reach = pairs
        pairs = int(reach.sum().item())
        mean_deg = g.nnz / g.n
        line.update({"metric": "BFS per second and GTEPS (aggregate), all-source closeness",
                     "value": count / (ms * 1e-3), "unit": "BFS/s", "ms_per_step": ms,
                     "gteps_est": pairs * mean_deg / 2 / (ms * 1e-3) / 1e9,
                     "config": {"workload": args.workload, "graph": desc, "n": g.n, "nnz": g.nnz,
                                "sources": count, "batch": 1024, "tau": h.info()["tau"]},
                     "full_run_estimate_s": (g.n / count) * ms * 1e-3,
                     "gpu_launches": (count + 1023) // 1024})
    elif args.workload == "switch_heldout":
        line.update(run_heldout(args, torch, blest, dev, stream))
    else:
        b = gg.ba_batch(10000, 1000, 100000, 4, seed=3)
        srcs = np.zeros(b.g, np.int32)            # vertex 0 of every graph
        h = blest.build_many(b)
        h.set_stream(stream.cuda_stream, True)
        out = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device=dev)
        for _ in range(args.warmup):
            h.bfs_many(srcs, out)
        h.sync()
        a, e = _events(torch)
        a.record(stream)
        for _ in range(args.steps):
            h.bfs_many(srcs, out)
        e.record(stream)
        torch.cuda.synchronize()
        h.sync()
        ms = a.elapsed_time(e) / args.steps
        # traversed arcs: out-degrees of the reached vertices of every graph
        degs = np.concatenate([np.diff(b.row_ptr[b.vtx_off[i] + i: b.vtx_off[i + 1] + i + 1]) for i in range(b.g)])
        reached = (out >= 0).cpu().numpy()
        arcs = int(degs[reached].sum())
        line.update({"metric": "GTEPS (aggregate), batched BFS over 10,000 BA graphs", "value": arcs / 2 / (ms * 1e-3) / 1e9,
                     "unit": "GTEPS", "ms_per_step": ms,
                     "config": {"workload": args.workload,
                                "graph": "10,000 Barabasi-Albert graphs, n log-uniform in [1e3, 1e5], m = 4",
                                "total_vertices": int(b.vtx_off[-1]), "total_arcs": arcs, "source": "vertex 0"},
                     "gpu_launches": args.steps})
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_heldout(args, torch, blest, dev, stream):
    """The learned level-mode policy on graph families it was not trained on
    (RMAT scale 25, Barabasi-Albert 2^24 m = 8, random geometric 2^24 with
    average degree 10): per-level device times of every mode give the time
    regret of the learned policy and of the paper's rule against the
    per-level optimum; whole-BFS GTEPS of both policies on the same sources."""
    from paper_2606_05081_gb300 import switch
    w = switch.load_weights()
    if w is None:
        return {"metric": "switching regret", "value": None, "unavailable": "no trained weights"}
    fams = [("rmat25", lambda: gg.rmat(25, 16, seed=25), "RMAT scale 25, edge factor 16"),
            ("ba16m_m8", lambda: gg.ba(1 << 24, 8, seed=26), "Barabasi-Albert, 2^24 vertices, m = 8"),
            ("rgg16m", lambda: gg.rgg(1 << 24, 10.0, seed=27), "random geometric, 2^24 points, average degree 10")]
    per, regs = {}, []
    for name, mk, desc in fams:
        g = mk()
        srcs = gg.sources(g, args.sources, 5)
        h = blest.build(g.n, g.row_ptr, g.col)
        h.set_stream(stream.cuda_stream, True)
        h.load_model(w)
        ev = switch.evaluate(h, srcs[:8], w, reps=2)
        deg = np.diff(g.row_ptr)
        out = torch.empty(g.n, dtype=torch.int32, device=dev)
        rates = {}
        for pol, tc in (("learned", False), ("heuristic", True)):
            h.set_engine(tc)
            h.set_policy(blest.POLICY_LEARNED if pol == "learned" else blest.POLICY_HEURISTIC)
            r = []
            for s in srcs:
                h.bfs(int(s), out)
                h.sync()
                a, b = _events(torch)
                a.record(stream)
                h.bfs(int(s), out)
                b.record(stream)
                torch.cuda.synchronize()
                h.sync()
                lv = out.cpu().numpy()
                r.append(deg[lv >= 0].sum() / 2 / (a.elapsed_time(b) * 1e-3) / 1e9)
            rates[pol] = harmonic(r)
        per[name] = {"graph": desc, "n": g.n, "nnz": g.nnz, "regret_learned": ev["regret_learned"],
                     "regret_heuristic_tc": ev["regret_heuristic_tc"], "regret_heuristic_cc": ev["regret_heuristic_cc"],
                     "ms_learned": ev["ms_learned"], "ms_heuristic_tc": ev["ms_heuristic_tc"],
                     "ms_optimal": ev["ms_optimal"], "gteps_learned": rates["learned"],
                     "gteps_heuristic_tc": rates["heuristic"]}
        regs.append(ev["regret_learned"])
        h.close()
        del g
    return {"metric": "switching regret of the learned policy (held-out families), mean", "value": float(np.mean(regs)),
            "unit": "fraction over the per-level optimum", "higher_is_better": False,
            "config": {"workload": "switch_heldout", "sources": args.sources, "regret_sources": 8},
            "per_family": per, "gpu_launches": None}


if __name__ == "__main__":
    main()
