"""Pins for the reordering oracles (CPU only): RCM (§4.2) and
JaccardWithWindows (§4.1, Algorithm 1)."""
import numpy as np
import pytest

import graphgen as gg
from oracle import reorder


def _is_perm(p, n):
    return np.array_equal(np.sort(p), np.arange(n))


@pytest.mark.parametrize("n", [2, 9, 100])
def test_rcm_path_closed_form(n):
    """Both ends of a path have degree 1; CM starts at vertex 0 and walks the
    path, so the reversed order puts vertex v at n-1-v."""
    assert np.array_equal(reorder.rcm(gg.path(n)), n - 1 - np.arange(n))


def test_rcm_star_closed_form():
    """Star: CM starts at leaf 1 (degree 1, lowest id), then the centre, then
    leaves 2..n-1 by id; reversed."""
    n = 12
    p = reorder.rcm(gg.star(n))
    expect = np.empty(n, np.int64)
    expect[1], expect[0] = n - 1, n - 2
    expect[2:] = n - 1 - np.arange(2, n)
    assert np.array_equal(p, expect)


def test_rcm_is_a_bfs_order_and_narrows_a_scrambled_lattice():
    R, C = 30, 40
    lat = gg.lattice(R, C)
    scr = np.random.RandomState(3).permutation(R * C)
    g = reorder.permute(lat, scr)
    p = reorder.rcm(g)
    assert _is_perm(p, g.n)
    # CM order (reverse of RCM) visits vertices level by level from its start
    order = np.empty(g.n, np.int64)
    order[g.n - 1 - p] = np.arange(g.n)
    import oracle
    lv = oracle.bfs(g, int(order[0]))
    assert np.all(np.diff(lv[order]) >= 0)
    # bandwidth comparable to the natural row-major order (C) and to SciPy's RCM
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    m = sp.csr_matrix((np.ones(g.nnz), g.col, g.row_ptr), shape=(g.n, g.n))
    sp_order = reverse_cuthill_mckee(m, symmetric_mode=True)
    sp_p = np.empty(g.n, np.int64)
    sp_p[sp_order] = np.arange(g.n)
    assert reorder.bandwidth(g, p) <= 2 * min(R, C) + 2
    assert reorder.bandwidth(g, p) <= 1.5 * reorder.bandwidth(g, sp_p) + 2
    assert reorder.bandwidth(g, scr) > 10 * min(R, C)  # the scrambled input was wide


def test_rcm_components_and_isolated():
    g = gg.disjoint_union(gg.path(5), gg.from_edges(2, [], [], True), gg.cycle(6))
    p = reorder.rcm(g)
    assert _is_perm(p, g.n)
    # the isolated vertices (degree 0) start the CM order, so they end the RCM order
    assert sorted(p[[5, 6]].tolist()) == [g.n - 2, g.n - 1]


@pytest.mark.parametrize("maker,W", [(lambda: gg.rmat(8, seed=1), 64), (lambda: gg.ba(300, 3, seed=2), 96),
                                     (lambda: gg.grid(12, 20, seed=3), 80), (lambda: gg.rmat(9, seed=4), 512),
                                     (lambda: gg.star(70), 32)])
def test_jaccard_incremental_equals_recompute(maker, W):
    g = maker()
    a = reorder.jaccard_with_windows(g, 8, W)
    b = reorder.jaccard_greedy_recompute(g, 8, W)
    assert np.array_equal(a, b)
    assert _is_perm(a, g.n)


def test_jaccard_keeps_columns_in_their_window():
    g = gg.rmat(11, seed=6)
    W = 256
    p = reorder.jaccard_with_windows(g, 8, W)
    assert np.array_equal(np.arange(g.n) // W, p // W)


def test_jaccard_planted_communities():
    """64 groups of 8 columns with identical neighbourhoods (complete
    bipartite to their own group of 8 vertices in the other window): every
    slice set built by Algorithm 1 is exactly one group."""
    rs = np.random.RandomState(0)
    W, K = 512, 64
    cols = rs.permutation(W).reshape(K, 8)
    rows = (W + rs.permutation(W)).reshape(K, 8)
    u, v = [], []
    for k in range(K):
        for a in cols[k]:
            for b in rows[k]:
                u.append(a)
                v.append(b)
    g = gg.from_edges(2 * W, u, v, symmetrize=True)
    p = reorder.jaccard_with_windows(g, 8, W)
    for groups in (cols, rows):
        sets = {frozenset(int(x) for x in p[grp] // 8) for grp in groups}
        assert all(len(s) == 1 for s in sets)            # one slice set per group
        assert len(sets) == K


def test_jaccard_compresses_vs_random_order():
    """On an RMAT graph the Jaccard order needs fewer slices than a random
    order (the purpose of §4.1)."""
    import oracle
    g = gg.rmat(11, seed=8)
    rnd = np.random.RandomState(1).permutation(g.n)
    gr = reorder.permute(g, rnd)
    pj = reorder.jaccard_with_windows(gr, 8, 512)
    s_rand = oracle.bvss(gr, 8)["num_slices"]
    s_jacc = oracle.bvss(reorder.permute(gr, pj), 8)["num_slices"]
    assert s_jacc < 0.95 * s_rand


def test_symmetrized_pattern():
    import graphgen as gg
    g = gg.from_edges(5, [0, 0, 1, 3, 4, 2], [1, 1, 2, 3, 2, 4], symmetrize=False)
    s = reorder.symmetrized(g)
    nb = [sorted(s.col[s.row_ptr[v]:s.row_ptr[v + 1]].tolist()) for v in range(5)]
    assert nb == [[1], [0, 2], [1, 4], [], [2]]      # 3->3 dropped, 0->1 once, 2<->4 once
    # an undirected graph is its own symmetrised pattern
    u = gg.rmat(9, seed=4)
    su = reorder.symmetrized(u)
    assert np.array_equal(su.row_ptr, u.row_ptr) and np.array_equal(su.col, u.col)
    # on a directed graph, RCM of the pattern is a permutation
    d = gg.er(300, 900, seed=2, directed=True)
    p = reorder.rcm(reorder.symmetrized(d))
    assert np.array_equal(np.sort(p), np.arange(300))
