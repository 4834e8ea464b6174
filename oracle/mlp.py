"""CPU oracle (fp64) of the per-level kernel-choice MLP.  TEST
INFRASTRUCTURE ONLY.

The paper chooses the level mode with a hand-set rule (§5.3 Eq. 5 with
eta = 10, calibrated for Hopper, §7.1); the learned policy replaces it with a
3-layer perceptron that predicts, from six per-level features, the log
device time of each of nine level choices (the five level modes, lazy ones
with one VSS pass in flight, plus lazy CUDA-core and b1-MMA levels with two
and four passes), and picks the smallest.

Network (same layout as the device weights): x = (raw - mean) * istd;
h1 = tanh(W1 x + b1) (32); h2 = tanh(W2 h1 + b2) (32); y = W3 h2 + b3 (9).
Loss: mean over the observed (sample, mode) pairs of (y - log t)^2.
Optimiser: Adam (Kingma & Ba, 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

IN, H, OUT = 6, 32, 9
OFF_MEAN, OFF_ISTD = 0, 6
OFF_W1 = 12
OFF_B1 = OFF_W1 + H * IN
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + OUT * H
NW = OFF_B3 + OUT


def raw_features(frontier, fedges, unvisited, slots, level, avg_deg):
    """The six inputs: log1p of frontier vertices, frontier out-arcs,
    unvisited vertices, active BVSS slots (tau per scheduled VSS), level
    index and average degree."""
    return np.stack([np.log1p(np.asarray(frontier, np.float64)),
                     np.log1p(np.asarray(fedges, np.float64)),
                     np.log1p(np.maximum(np.asarray(unvisited, np.float64), 0)),
                     np.log1p(np.asarray(slots, np.float64)),
                     np.log1p(np.asarray(level, np.float64)),
                     np.log1p(np.broadcast_to(np.asarray(avg_deg, np.float64), np.shape(frontier)))], axis=-1)


def unpack(w):
    w = np.asarray(w, np.float64)
    return dict(mean=w[OFF_MEAN:OFF_MEAN + IN], istd=w[OFF_ISTD:OFF_ISTD + IN],
                W1=w[OFF_W1:OFF_B1].reshape(H, IN), b1=w[OFF_B1:OFF_W2],
                W2=w[OFF_W2:OFF_B2].reshape(H, H), b2=w[OFF_B2:OFF_W3],
                W3=w[OFF_W3:OFF_B3].reshape(OUT, H), b3=w[OFF_B3:NW])


def init_weights(mean, std, seed: int = 0) -> np.ndarray:
    """Glorot-uniform layers, zero biases, normalisation from the data."""
    rs = np.random.RandomState(seed)
    w = np.zeros(NW, np.float64)
    w[OFF_MEAN:OFF_MEAN + IN] = mean
    w[OFF_ISTD:OFF_ISTD + IN] = 1.0 / np.maximum(std, 1e-6)
    for off, fo, fi in ((OFF_W1, H, IN), (OFF_W2, H, H), (OFF_W3, OUT, H)):
        a = np.sqrt(6.0 / (fi + fo))
        w[off:off + fo * fi] = rs.uniform(-a, a, fo * fi)
    return w


def forward(w, raw):
    p = unpack(w)
    x = (np.asarray(raw, np.float64) - p["mean"]) * p["istd"]
    h1 = np.tanh(x @ p["W1"].T + p["b1"])
    h2 = np.tanh(h1 @ p["W2"].T + p["b2"])
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, h1, h2)


def loss_and_grad(w, raw, target, mask):
    """Masked mean squared error and its gradient with respect to every
    trainable parameter (the normalisation entries get zero gradient)."""
    p = unpack(w)
    y, (x, h1, h2) = forward(w, raw)
    m = np.asarray(mask, np.float64)
    cnt = max(m.sum(), 1.0)
    r = (y - np.asarray(target, np.float64)) * m
    loss = float((r * r).sum() / cnt)
    dy = 2.0 * r / cnt                               # [N, OUT]
    g = np.zeros(NW, np.float64)
    g[OFF_W3:OFF_B3] = (dy.T @ h2).ravel()
    g[OFF_B3:NW] = dy.sum(0)
    dh2 = dy @ p["W3"]
    da2 = dh2 * (1.0 - h2 * h2)
    g[OFF_W2:OFF_B2] = (da2.T @ h1).ravel()
    g[OFF_B2:OFF_W3] = da2.sum(0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (1.0 - h1 * h1)
    g[OFF_W1:OFF_B1] = (da1.T @ x).ravel()
    g[OFF_B1:OFF_W2] = da1.sum(0)
    return loss, g


def adam_step(w, g, m, v, t, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
    """One Adam step (t counts from 1); normalisation entries are frozen.
    wd adds an L2 penalty (wd/2)|w|^2 of the trainable entries to the loss,
    i.e. wd * w to their gradient."""
    g = np.asarray(g, np.float64).copy()
    g[OFF_W1:] += wd * np.asarray(w, np.float64)[OFF_W1:]
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    w = w.copy()
    w[OFF_W1:] -= lr * mh[OFF_W1:] / (np.sqrt(vh[OFF_W1:]) + eps)
    return w, m, v


BU_GUARD_LOG = np.log(16.0)


def choose(w, raw):
    """Choice with the smallest predicted log time (lowest index on ties);
    bottom-up (choice 4) is excluded on levels with more than 16 unvisited
    vertices per out-arc of the frontier (raw features 2 and 1): a
    bottom-up level reads every unvisited vertex, a top-down level the
    frontier's arcs."""
    y, _ = forward(w, raw)
    raw = np.atleast_2d(np.asarray(raw, np.float64))
    y = np.array(y, np.float64, copy=True).reshape(raw.shape[0], OUT)
    y[raw[:, 2] > raw[:, 1] + BU_GUARD_LOG, 4] = np.inf
    return np.argmin(y, axis=-1)


def heuristic_choose(lazy, tc, switching, eta, unvisited, queue):
    """The paper's rule (§5.3, §7.1): lazy or eager by U_div (per graph),
    bottom-up when switching is enabled and #unvisited < eta * |Q|."""
    td = (3 if tc else 2) if lazy else (1 if tc else 0)
    u = np.asarray(unvisited, np.float64)
    q = np.asarray(queue, np.float64)
    out = np.full(u.shape, td, np.int64)
    if switching:
        out[u < eta * q] = 4
    return out


def regret(times, chosen):
    """sum_l t(chosen_l) / sum_l min_mode t(l) - 1 over levels with a full
    time row (the per-level optimum of the switching analysis of §7.1)."""
    t = np.asarray(times, np.float64)
    c = np.asarray(chosen, np.int64)
    got = t[np.arange(len(c)), c].sum()
    best = t.min(axis=1).sum()
    return float(got / best - 1.0)
