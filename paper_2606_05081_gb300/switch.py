"""Learned per-level kernel switch: data collection, training, evaluation.

Because the BFS state after a level (levels, visited and frontier bits,
queues) is the same whichever mode ran it, one BFS per fixed mode gives the
device time of every mode at every level of that BFS.  Those per-level
times, logged by the persistent kernel (globaltimer at each level barrier),
are the training targets; the features are the six per-level counters the
kernel itself feeds to the network.  Training runs on the GPU
(blest_mlp_train); the heuristic of §5.3 / §7.1 is the baseline, and the
time regret of a policy is sum_l t(chosen_l) / sum_l min_mode t(l) - 1 (the
per-level optimum of the paper's switching analysis, §7.1).

    python -m paper_2606_05081_gb300.switch train [--out PATH]

trains on the standard training graphs (RMAT scales 14-24, road-like
grids, Barabasi-Albert graphs), each built with the warp-wide (tau = 128)
and the narrow (tau = 32) sigma = 8 VSS, and writes the weights next to
this file.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

from . import (MLP_NW, NUM_CHOICES, POLICY_FIXED, POLICY_HEURISTIC, Graph, choice_mode_batch,
               choice_of, mlp_features, mlp_predict, mlp_train)

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "switch_mlp.f32")
def level_times(h: Graph, source: int, out, reps: int = 1):
    """Per-level records of one BFS and its (levels x choices) device-time
    matrix in ns (min over reps): choice c runs its mode at every level with
    its number of VSS passes in flight."""
    recs, T = None, None
    info = h.info()
    block, batch0 = info["block_threads"], info["vss_batch"]
    for c in range(NUM_CHOICES):
        mode, batch = choice_mode_batch(c)
        h.set_launch(block, batch)
        h.set_policy(POLICY_FIXED, mode)
        best = None
        for _ in range(reps):
            h.bfs(int(source), out)
            log = h.level_log()
            t = np.array([r["t_ns"] for r in log], np.float64)
            best = t if best is None else np.minimum(best, t)
            if recs is None:
                recs = log
        if T is None:
            T = np.zeros((len(best), NUM_CHOICES))
        if len(best) != T.shape[0]:
            raise RuntimeError("level count differs between modes")
        T[:, c] = best
    h.set_launch(block, batch0)
    h.set_policy(POLICY_HEURISTIC)
    return recs, T


def dataset(handles, sources_per, reps: int = 2, avg_degs=None):
    """Features (n, 6), log-time targets (n, NUM_CHOICES), mask, and the raw
    matrices."""
    import torch
    X, Y, mats = [], [], []
    for i, (h, srcs) in enumerate(zip(handles, sources_per)):
        out = torch.empty(h.n, dtype=torch.int32, device="cuda")
        info = h.info()
        ad = (avg_degs[i] if avg_degs else info["nnz"] / info["n"])
        for s in srcs:
            recs, T = level_times(h, int(s), out, reps)
            X.append(mlp_features(recs, ad))
            Y.append(np.log(np.maximum(T, 1.0)))
            mats.append((recs, T))
    X = np.concatenate(X).astype(np.float32)
    Y = np.concatenate(Y).astype(np.float32)
    return X, Y, np.ones_like(Y), mats


def init_weights(X, seed: int = 0) -> np.ndarray:
    rs = np.random.RandomState(seed)
    w = np.zeros(MLP_NW, np.float32)
    w[0:6] = X.mean(0)
    w[6:12] = 1.0 / np.maximum(X.std(0), 1e-3)
    off = 12
    for fo, fi in ((32, 6), (32, 32), (NUM_CHOICES, 32)):
        a = np.sqrt(6.0 / (fi + fo))
        w[off:off + fo * fi] = rs.uniform(-a, a, fo * fi)
        off += fo * fi + fo
    return w


def train(X, Y, M=None, epochs: int = 1500, lr: float = 5e-3, weight_decay: float = 3e-3, seed: int = 0):
    """Targets are each mode's log time relative to the level's best mode
    (only the argmin matters); each level is weighted by the square root of
    its best time, so the expensive levels the regret is made of dominate;
    an L2 penalty keeps the predictions smooth on graph families outside the
    training set."""
    Y = np.asarray(Y, np.float32)
    rel = Y - Y.min(axis=1, keepdims=True)
    tmin = np.exp(Y.min(axis=1).astype(np.float64))
    wt = np.sqrt(tmin / tmin.mean()).astype(np.float32)
    mask = np.repeat(wt[:, None], Y.shape[1], axis=1)
    if M is not None:
        mask = mask * np.asarray(M, np.float32)
    w0 = init_weights(X, seed)
    return mlp_train(X, rel, mask, w0, epochs, lr, weight_decay)


def heuristic_modes(info: dict, recs, eta: float = 10.0, tc: bool = False, batch: int = 2):
    """The paper's rule on logged levels (§5.3, §7.1), as choices (its lazy
    levels run with the launch's `batch` VSS passes in flight)."""
    lazy, sw = info["lazy"], info["switching"]
    out = []
    for r in recs:
        m = (3 if tc else 2) if lazy else (1 if tc else 0)
        if sw and r["unvisited"] < eta * r["queue"]:
            m = 4
        out.append(choice_of(m, batch))
    return np.array(out)


def regret(T, chosen) -> float:
    T = np.asarray(T, np.float64)
    c = np.asarray(chosen, np.int64)
    return float(T[np.arange(len(c)), c].sum() / T.min(axis=1).sum() - 1.0)


def evaluate(h: Graph, sources, weights, reps: int = 2):
    """Regret of the heuristic and of the MLP on measured per-level times."""
    import torch
    out = torch.empty(h.n, dtype=torch.int32, device="cuda")
    info = h.info()
    ad = info["nnz"] / info["n"]
    tot = {"heuristic_tc": 0.0, "heuristic_cc": 0.0, "learned": 0.0, "optimal": 0.0}
    for s in sources:
        recs, T = level_times(h, int(s), out, reps)
        _, ch = mlp_predict(weights, mlp_features(recs, ad))
        r = np.arange(len(ch))
        tot["heuristic_tc"] += T[r, heuristic_modes(info, recs, tc=True, batch=info["vss_batch"])].sum()
        tot["heuristic_cc"] += T[r, heuristic_modes(info, recs, tc=False, batch=info["vss_batch"])].sum()
        tot["learned"] += T[r, ch].sum()
        tot["optimal"] += T.min(axis=1).sum()
    opt = tot["optimal"]
    return {"regret_heuristic_tc": tot["heuristic_tc"] / opt - 1.0,
            "regret_heuristic_cc": tot["heuristic_cc"] / opt - 1.0,
            "regret_learned": tot["learned"] / opt - 1.0,
            "ms_heuristic_tc": tot["heuristic_tc"] / 1e6, "ms_heuristic_cc": tot["heuristic_cc"] / 1e6,
            "ms_learned": tot["learned"] / 1e6, "ms_optimal": opt / 1e6}


def load_weights(path: str = DEFAULT_WEIGHTS):
    if not os.path.exists(path):
        return None
    w = np.fromfile(path, dtype=np.float32)
    return w if w.size == MLP_NW else None


def save_weights(w, path: str = DEFAULT_WEIGHTS, meta: dict | None = None):
    np.asarray(w, np.float32).tofile(path)
    if meta is not None:
        with open(os.path.splitext(path)[0] + ".json", "w") as f:
            json.dump(meta, f, indent=1)


TRAIN_LAYOUTS = ((8, 128), (8, 32))


def training_graphs():
    """The graph families of the single-source (RMAT, road-like grid) and
    batched (RMAT, Barabasi-Albert with m = 4 and 8) workloads over the size
    range they are used at; random geometric graphs are left out (a held-out
    family), as are RMAT 25 and Barabasi-Albert graphs of 2^24 vertices."""
    import graphgen as gg
    out = [(f"rmat{s}", (lambda s=s: gg.rmat(s, 16, seed=100 + s)), {}) for s in (14, 16, 18, 20, 22, 24)]
    out += [(f"grid{r}", (lambda r=r: gg.grid(r, r, 0.05, 0.001, seed=200 + r)), {"reorder": 1})
            for r in (256, 1024, 2048)]
    out += [(f"ba{n}", (lambda n=n: gg.ba(n, 4, seed=300 + n % 997)), {}) for n in (1 << 16, 1 << 20, 1 << 22)]
    out += [(f"ba{n}m8", (lambda n=n: gg.ba(n, 8, seed=400 + n % 991)), {}) for n in (1 << 20, 1 << 22)]
    return out


def main(argv=None):
    import argparse

    import graphgen as gg
    import torch

    from . import build
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train"])
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--sources", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=3000)
    args = ap.parse_args(argv)
    torch.cuda.init()
    t0 = time.time()
    Xs, Ys, names = [], [], []
    for name, make, opts in training_graphs():
        g = make()
        srcs = gg.sources(g, args.sources, 100)
        for sigma, tau in TRAIN_LAYOUTS:
            h = build(g.n, g.row_ptr, g.col, sigma=sigma, tau=tau, **opts)
            X, Y, M, _ = dataset([h], [srcs])
            Xs.append(X)
            Ys.append(Y)
            names.append((f"{name}_s{sigma}t{tau}", int(len(X))))
            h.close()
            print(f"collected {name} sigma {sigma} tau {tau}: {len(X)} levels", file=sys.stderr)
    X = np.concatenate(Xs)
    Y = np.concatenate(Ys)
    w, hist = train(X, Y, np.ones_like(Y), epochs=args.epochs)
    meta = {"graphs": names, "samples": int(len(X)), "epochs": args.epochs, "loss_first": float(hist[0]),
            "loss_last": float(hist[-1]), "seconds": round(time.time() - t0, 1)}
    save_weights(w, args.out, meta)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
