"""Pins of the scale-free-like classifier oracle (§4.2 footnote) on hand-built
degree sequences whose answers follow from the definition by hand, and
on graph families whose character is known (a lattice is not scale-free,
a star and a Barabasi-Albert graph are)."""
import math

import numpy as np
import pytest

import graphgen as gg
from oracle import classify


def test_regular_degrees_are_not_heavy_tailed():
    r = classify.heavy_tailed(np.full(1000, 4))
    # top 1 % = 10 vertices hold exactly 1 %, top 10 % exactly 10 %; no k >= 5 to fit
    assert r["top1"] == pytest.approx(0.01) and r["top10"] == pytest.approx(0.10)
    assert r["points"] == 0 and not r["powerlaw"] and not r["heavy"]


def test_top_shares_by_hand():
    # 200 vertices: two of degree 100, eighteen of degree 10, 180 of degree 1
    deg = np.array([100] * 2 + [10] * 18 + [1] * 180)
    t1, t10 = classify.concentration(deg)
    tot = 200 + 180 + 180
    assert t1 == 200 / tot                     # floor(200/100) = 2 vertices
    assert t10 == (200 + 180) / tot            # floor(200/10) = 20 vertices
    assert classify.heavy_tailed(deg)["concentrated"]
    # top-1% set is never empty: 50 vertices -> one vertex
    assert classify.concentration(np.array([10] + [1] * 49))[0] == 10 / 59


def test_concentration_thresholds_are_inclusive_and_both_needed():
    # n = 1000, total 10,000: the top 10 vertices hold 500 (exactly 5 %), the
    # top 100 hold 4,000 (exactly 40 %)
    deg = np.array([50] * 10 + [39] * 80 + [38] * 10 + [7] * 600 + [6] * 300)
    assert deg.sum() == 10000
    t1, t10 = classify.concentration(deg)
    assert t1 == 0.05 and t10 == 0.40
    assert classify.heavy_tailed(deg)["concentrated"]
    below1 = deg.copy()
    below1[0] -= 1       # top 1 % just under 5 % (same total)
    below1[-1] += 1
    assert not classify.heavy_tailed(below1)["concentrated"]
    below10 = deg.copy()
    below10[99] -= 1     # top 10 % just under 40 %, top 1 % unchanged
    below10[-1] += 1
    assert classify.concentration(below10)[0] == 0.05
    assert not classify.heavy_tailed(below10)["concentrated"]


def test_exact_power_law_histogram_gives_gamma_and_r2_one():
    # h(k) = 2^20 / k^2 for k = 2^j, j = 3..10: exact integers, slope -2 in log-log
    deg = []
    for j in range(3, 11):
        k = 1 << j
        deg += [k] * ((1 << 20) // (k * k))
    gamma, r2, pts = classify.powerlaw_fit(deg)
    assert pts == 8 and gamma == pytest.approx(2.0, abs=1e-12) and r2 == pytest.approx(1.0, abs=1e-12)
    # the points below k = 5 are not part of the fit
    gamma2, _, pts2 = classify.powerlaw_fit(deg + [1] * 100000 + [4] * 3)
    assert pts2 == 8 and gamma2 == pytest.approx(2.0, abs=1e-12)


def test_two_point_fit_by_hand():
    # h(5) = 100, h(10) = 25: slope = log(25/100) / log(10/5) = -2; two points fit exactly
    deg = [5] * 100 + [10] * 25
    gamma, r2, pts = classify.powerlaw_fit(deg)
    assert pts == 2 and gamma == pytest.approx(2.0) and r2 == pytest.approx(1.0)
    assert classify.heavy_tailed(deg)["powerlaw"]
    # one point only: no fit
    assert math.isnan(classify.powerlaw_fit([7] * 9)[0])


def test_power_law_test_alone_can_decide():
    # a power-law tail (gamma 3) under a dominant block of degree-4 vertices:
    # concentration fails, the fit over k >= 5 succeeds
    deg = [4] * 1_000_000
    for k in range(5, 61):
        deg += [k] * int(1e6 * k ** -3.0)
    r = classify.heavy_tailed(deg)
    assert not r["concentrated"]
    assert r["powerlaw"] and 2.8 < r["gamma"] < 3.2 and r["r2"] > 0.95 and r["heavy"]


def test_power_law_outside_the_gamma_range_or_poor_fit_fails():
    steep = []
    for k in range(5, 12):
        steep += [k] * int(1e9 * k ** -6.0)     # gamma 6 > 5
    r = classify.heavy_tailed(steep)
    assert r["gamma"] > 5 and not r["powerlaw"]
    flat = []
    for k in range(5, 200):
        flat += [k] * 3                          # slope 0: gamma 0 < 1
    assert not classify.heavy_tailed(flat)["powerlaw"]
    rng = np.random.default_rng(1)
    noisy = []
    for k in range(5, 400):
        noisy += [k] * int(rng.integers(1, 50))  # no trend: R^2 near 0
    r = classify.heavy_tailed(noisy)
    assert r["r2"] < 0.70 and not r["powerlaw"]


def test_in_degrees_alone_can_make_a_directed_graph_scale_free():
    # a directed in-star: out-degrees all 1 (not heavy), in-degrees one hub
    n = 500
    out_deg = np.ones(n, np.int64)
    out_deg[0] = 0
    in_deg = np.zeros(n, np.int64)
    in_deg[0] = n - 1
    r = classify.scale_free_like(out_deg, in_deg)
    assert not r["out"]["heavy"] and r["in"]["heavy"] and r["scale_free"]


def test_known_families():
    assert not classify.scale_free_like(*classify.degrees(gg.lattice(64, 64)))["scale_free"]
    assert not classify.scale_free_like(*classify.degrees(gg.grid(128, 128, 0.05, 0.001, seed=1)))["scale_free"]
    assert classify.scale_free_like(*classify.degrees(gg.star(300)))["scale_free"]
    assert classify.scale_free_like(*classify.degrees(gg.rmat(14, seed=1)))["scale_free"]
    ba = classify.scale_free_like(*classify.degrees(gg.ba(1 << 15, 4, seed=2)))
    assert ba["scale_free"]
    assert 2.0 < ba["out"]["gamma"] < 3.5       # preferential attachment: gamma near 3


def test_degrees_drop_duplicates_and_loops():
    g = gg.from_edges(4, [0, 0, 1, 2, 2], [1, 1, 1, 3, 0], symmetrize=False)
    out_deg, in_deg = classify.degrees(g)
    assert list(out_deg) == [1, 0, 2, 0] and list(in_deg) == [1, 1, 0, 1]
