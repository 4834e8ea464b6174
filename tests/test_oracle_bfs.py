"""Pins for the BFS-level and closeness oracle (CPU only).

Each check fixes the oracle to something other than itself: closed forms on
graphs whose distances are known, Floyd-Warshall on tiny graphs, SciPy's
shortest-path routine, and the BFS edge invariant.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import graphgen as gg
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _scipy_levels(g, src):
    m = sp.csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    d = csg.shortest_path(m, directed=True, unweighted=True, indices=[src])[0]
    out = np.where(np.isinf(d), -1, d).astype(np.int64)
    return out


def _floyd_warshall(g):
    n = g.n
    INF = 10 ** 9
    d = np.full((n, n), INF, np.int64)
    np.fill_diagonal(d, 0)
    for v in range(n):
        for w in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
            d[v, w] = min(d[v, w], 1)
    for k in range(n):
        d = np.minimum(d, d[:, k:k + 1] + d[k:k + 1, :])
    return np.where(d >= INF, -1, d)


@pytest.mark.parametrize("n", [1, 2, 7, 64, 1000])
def test_path_closed_form(n):
    g = gg.path(n) if n > 1 else gg.from_edges(1, [], [], True)
    for s in {0, n // 2, n - 1}:
        assert np.array_equal(oracle.bfs(g, s), np.abs(np.arange(n) - s))


@pytest.mark.parametrize("n", [3, 10, 257])
def test_cycle_closed_form(n):
    g = gg.cycle(n)
    for s in (0, n // 3):
        k = np.abs(np.arange(n) - s)
        assert np.array_equal(oracle.bfs(g, s), np.minimum(k, n - k))


def test_star_and_complete():
    n = 50
    st = gg.star(n)
    lv = oracle.bfs(st, 0)
    assert lv[0] == 0 and np.all(lv[1:] == 1)
    lv = oracle.bfs(st, 7)
    assert lv[7] == 0 and lv[0] == 1 and np.all(np.delete(lv, [0, 7]) == 2)
    kn = gg.complete(33)
    lv = oracle.bfs(kn, 5)
    assert lv[5] == 0 and np.all(np.delete(lv, 5) == 1)


@pytest.mark.parametrize("rows,cols", [(1, 9), (17, 23), (64, 64)])
def test_lattice_manhattan(rows, cols):
    g = gg.lattice(rows, cols)
    r, c = np.divmod(np.arange(rows * cols), cols)
    for s in (0, (rows // 2) * cols + cols // 3, rows * cols - 1):
        sr, sc = divmod(s, cols)
        assert np.array_equal(oracle.bfs(g, s), np.abs(r - sr) + np.abs(c - sc))


def test_unreached_components_are_minus_one():
    g = gg.disjoint_union(gg.path(10), gg.cycle(7), gg.from_edges(3, [], [], True))
    lv = oracle.bfs(g, 3)
    assert np.all(lv[10:] == -1)
    assert np.array_equal(lv[:10], np.abs(np.arange(10) - 3))
    lv = oracle.bfs(g, 18)  # isolated vertex
    assert lv[18] == 0 and (lv >= 0).sum() == 1


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("directed", [False, True])
def test_floyd_warshall_tiny(seed, directed):
    n = [5, 17, 33, 64, 64, 48][seed]
    g = gg.er(n, 2 * n, seed=100 + seed, directed=directed)
    d = _floyd_warshall(g)
    for s in range(n):
        assert np.array_equal(oracle.bfs(g, s), d[s])


@pytest.mark.parametrize("maker", [lambda: gg.rmat(11, seed=3), lambda: gg.grid(40, 50, seed=4),
                                   lambda: gg.ba(3000, 3, seed=5), lambda: gg.rgg(3000, 8, seed=6),
                                   lambda: gg.er(2000, 3000, seed=8, directed=True)])
def test_scipy_shortest_path(maker):
    g = maker()
    srcs = gg.sources(g, 5, 11)
    lv = oracle.bfs_many(g, srcs)
    for k, s in enumerate(srcs):
        assert np.array_equal(lv[k], _scipy_levels(g, s))


def test_edge_invariant_rmat():
    g = gg.rmat(14, seed=1)
    srcs = gg.sources(g, 4, 1)
    src_of = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    for lv in oracle.bfs_many(g, srcs):
        a, b = lv[src_of], lv[g.col]
        assert np.all((a >= 0) == (b >= 0))
        both = a >= 0
        assert np.all(np.abs(a[both] - b[both]) <= 1)
        # every reached vertex but the source has a neighbour one level closer
        reached = np.flatnonzero(lv > 0)
        best = np.full(g.n, np.iinfo(np.int32).max)
        np.minimum.at(best, g.col, np.where(a >= 0, a, np.iinfo(np.int32).max))
        assert np.all(best[reached] == lv[reached] - 1)


def test_bfs_many_matches_single():
    g = gg.rmat(12, seed=2)
    srcs = gg.sources(g, 16, 3)
    lv = oracle.bfs_many(g, srcs, nthreads=4)
    for k, s in enumerate(srcs):
        assert np.array_equal(lv[k], oracle.bfs(g, s))


def test_invalid_source_raises():
    g = gg.path(4)
    with pytest.raises(ValueError):
        oracle.bfs(g, 4)
    with pytest.raises(ValueError):
        oracle.bfs(g, -1)


# ------------------------------------------------------------- closeness
def test_closeness_path_closed_form():
    n = 101
    far, reach, cc = oracle.closeness(gg.path(n))
    i = np.arange(n)
    assert np.array_equal(far, i * (i + 1) // 2 + (n - 1 - i) * (n - i) // 2)
    assert np.all(reach == n)
    assert np.array_equal(cc, (n - 1) / far.astype(np.float64))


def test_closeness_star_complete():
    n = 40
    far, reach, _ = oracle.closeness(gg.star(n))
    assert far[0] == n - 1 and np.all(far[1:] == 2 * n - 3)
    far, reach, cc = oracle.closeness(gg.complete(20))
    assert np.all(far == 19) and np.all(cc == 1.0)


def test_closeness_lattice_closed_form():
    R, C = 13, 9
    far, reach, _ = oracle.closeness(gg.lattice(R, C))
    r, c = np.divmod(np.arange(R * C), C)
    sr = np.abs(np.arange(R)[:, None] - np.arange(R)[None, :]).sum(1)
    sc = np.abs(np.arange(C)[:, None] - np.arange(C)[None, :]).sum(1)
    assert np.array_equal(far, C * sr[r] + R * sc[c])


def test_closeness_vs_scipy_and_disconnected():
    g = gg.disjoint_union(gg.rmat(9, seed=4), gg.path(30), gg.from_edges(2, [], [], True))
    far, reach, cc = oracle.closeness(g)
    m = sp.csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    d = csg.shortest_path(m, directed=False, unweighted=True)
    fin = np.isfinite(d)
    assert np.array_equal(far, np.where(fin, d, 0).sum(1).astype(np.int64))
    assert np.array_equal(reach, fin.sum(1))
    iso = np.flatnonzero(reach == 1)
    assert np.all(cc[iso] == 0.0)
    nz = far > 0
    assert np.array_equal(cc[nz], (reach[nz] - 1) / far[nz])


def test_far_reach_sample_equals_all():
    g = gg.grid(30, 30, seed=7)
    far, reach = oracle.far_reach(g)
    v = np.array([0, 17, 450, 899], np.int32)
    f2, r2 = oracle.far_reach(g, v)
    assert np.array_equal(f2, far[v]) and np.array_equal(r2, reach[v])


def test_gteps_edges():
    g = gg.path(10)
    assert oracle.gteps_edges(g, oracle.bfs(g, 0)) == 9
    g = gg.disjoint_union(gg.path(10), gg.complete(5))
    assert oracle.gteps_edges(g, oracle.bfs(g, 12)) == 10


def test_golden_fig1_bfs_step():
    """Fig. 1: vertex 3 has in-neighbours at columns 2, 4, 7 (1-indexed) of
    slice set 2; with the frontier on its 1st and 2nd columns, vertex 3 is
    discovered one level later."""
    gold = json.load(open(os.path.join(GOLD, "fig1_bvss_example.json")))
    cols = [16 + c - 1 for c in gold["vertex_3_in_neighbour_columns_1_indexed"]]
    g = gg.from_edges(24, cols, [3] * len(cols), symmetrize=False)
    front = [16 + i for i, ch in enumerate(gold["frontier_bits_of_slice_set_2"]) if ch == "1"]
    lv = oracle.bfs(g, front[1])
    assert lv[3] == 1
