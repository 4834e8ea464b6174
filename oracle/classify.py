"""CPU oracle of the scale-free-like test of the §4.2 footnote.  TEST
INFRASTRUCTURE ONLY (see the package header).

A graph is scale-free-like when its out- or its in-degree distribution is
heavy-tailed, and a distribution is heavy-tailed when either

  (a) concentration: the top 1 % of vertices by degree hold at least 5 % of
      the total degree and the top 10 % hold at least 40 %; or
  (b) power law: a least-squares line through the log-log degree histogram,
      over the degrees k >= 5, has slope -gamma with R^2 >= 0.70 and
      gamma in [1, 5].

Readings (the footnote fixes none of these):
  * "top p % of vertices" = the floor(p n / 100) vertices of highest degree,
    at least one;
  * the histogram is the exact count h(k) of vertices of degree k; the fit
    uses the points (log k, log h(k)) for every k >= 5 with h(k) > 0,
    unweighted, and needs at least two distinct points (else (b) fails);
  * R^2 = 1 - SS_res / SS_tot of that fit (the log base changes neither the
    slope nor R^2).
"""
from __future__ import annotations

import numpy as np


def concentration(deg) -> tuple[float, float]:
    """Shares of the total degree held by the top 1 % and top 10 % of the
    vertices (test (a)); (0, 0) when the total is 0."""
    d = np.sort(np.asarray(deg, dtype=np.int64))[::-1]
    n = len(d)
    tot = int(d.sum())
    if n == 0 or tot == 0:
        return 0.0, 0.0
    n1 = max(1, n // 100)
    n10 = max(1, n // 10)
    return float(d[:n1].sum()) / tot, float(d[:n10].sum()) / tot


def powerlaw_fit(deg, kmin: int = 5) -> tuple[float, float, int]:
    """(gamma, R^2, number of points) of the least-squares fit of log h(k)
    against log k over k >= kmin with h(k) > 0 (test (b)); gamma = slope
    negated.  Fewer than two points, or all at one k: (nan, nan, points)."""
    d = np.asarray(deg, dtype=np.int64)
    h = np.bincount(d) if len(d) else np.zeros(0, np.int64)
    ks = np.flatnonzero(h)
    ks = ks[ks >= kmin]
    if len(ks) < 2:
        return float("nan"), float("nan"), int(len(ks))
    x = np.log(ks.astype(np.float64))
    y = np.log(h[ks].astype(np.float64))
    slope, icpt = np.polyfit(x, y, 1)
    res = y - (slope * x + icpt)
    ss_res = float(np.sum(res * res))
    ss_tot = float(np.sum((y - y.mean()) ** 2))
    r2 = 1.0 - ss_res / ss_tot if ss_tot > 0 else float("nan")
    return float(-slope), r2, int(len(ks))


def heavy_tailed(deg) -> dict:
    """Both tests on one degree distribution."""
    t1, t10 = concentration(deg)
    gamma, r2, pts = powerlaw_fit(deg)
    conc = t1 >= 0.05 and t10 >= 0.40
    plaw = bool(np.isfinite(gamma) and np.isfinite(r2) and r2 >= 0.70 and 1.0 <= gamma <= 5.0)
    return {"top1": t1, "top10": t10, "gamma": gamma, "r2": r2, "points": pts,
            "concentrated": bool(conc), "powerlaw": plaw, "heavy": bool(conc or plaw)}


def scale_free_like(out_deg, in_deg=None) -> dict:
    """The footnote's decision: heavy-tailed out- or in-degrees (in_deg None:
    an undirected graph, whose in- and out-degrees coincide)."""
    o = heavy_tailed(out_deg)
    i = o if in_deg is None else heavy_tailed(in_deg)
    return {"out": o, "in": i, "scale_free": bool(o["heavy"] or i["heavy"])}


def degrees(g):
    """Out- and in-degrees of a CSR graph with duplicates and self loops
    removed (the graph the library reorders)."""
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    dst = g.col.astype(np.int64)
    keep = src != dst
    key = np.unique(src[keep] * n + dst[keep])
    out_deg = np.bincount(key // n, minlength=n)
    in_deg = np.bincount(key % n, minlength=n)
    return out_deg, in_deg
