"""Parity at the workloads' full sizes, on sampled outputs the oracle can
compute one by one (the oracle is a serial BFS, so full outputs at these
sizes would take hours on the host):

  * single-source: RMAT scale 24 with JaccardWithWindows (W = 2^16) and the
    4096 x 4096 road-like grid with RCM -- 16 sampled sources, whole level
    arrays compared, under the learned policy with the benchmark's default
    launch and under the paper's rule with the b1 MMA hit test;
  * multi-source: RMAT scale 22, 1024 lanes, stage 1 on CUDA cores and on
    the tcgen05 tensor cores -- 32 sampled lanes;
  * closeness: RMAT scale 18, all sources -- sampled targets (on an
    undirected graph the distance sum of a target is the level sum of a BFS
    from it); the 2048 x 2048 grid over two batches of sources -- sampled
    targets restricted to those sources;
  * 10,000 Barabasi-Albert graphs in one launch -- sampled graphs;
  * held-out families of the learned policy: RMAT scale 25, BA with 2^24
    vertices and m = 8, and a random geometric graph with 2^24 points and
    average degree 10 -- 16 sampled sources each.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def blest():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_05081_gb300 as b
    return b


def _check_sources(blest, h, g, srcs):
    from paper_2606_05081_gb300 import switch
    w = switch.load_weights()
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    refs = oracle.bfs_many(g, srcs)          # one serial BFS per source, all host cores
    arms = [(blest.POLICY_HEURISTIC, True)]
    if w is not None:
        h.load_model(w)
        arms.append((blest.POLICY_LEARNED, False))
    for policy, tc in arms:
        h.set_engine(tc)
        h.set_policy(policy)
        for s, ref in zip(srcs, refs):
            h.bfs(int(s), out)
            got = out.cpu().numpy()
            bad = np.flatnonzero(got != ref)
            assert len(bad) == 0, (policy, int(s), bad[:5])


def test_rmat24_jaccard_sampled_sources(blest):
    g = gg.rmat(24, 16, seed=2)
    with blest.build_graph(g, reorder=blest.REORDER_JACCARD, jaccard_window=65536) as h:
        p = h.perm()
        assert np.array_equal(np.sort(p), np.arange(g.n))
        assert np.array_equal(np.arange(g.n) // 65536, p // 65536)     # windows map onto themselves
        _check_sources(blest, h, g, gg.sources(g, 64, 7)[:16])


def test_grid4096_rcm_sampled_sources(blest):
    g = gg.grid(4096, 4096, 0.05, 0.001, seed=2)
    with blest.build_graph(g, reorder=blest.REORDER_RCM) as h:
        _check_sources(blest, h, g, gg.sources(g, 64, 7)[:16])


@pytest.mark.parametrize("engine", ["cuda_cores", "tcgen05"])
def test_msbfs_rmat22_1024_lanes_sampled(blest, engine):
    g = gg.rmat(22, 16, seed=3)
    srcs = gg.sources(g, 1024, 3)
    with blest.build_graph(g) as h:
        h.set_msbfs_engine(engine == "tcgen05")
        out = torch.empty((1024, g.n), dtype=torch.int32, device="cuda")
        h.msbfs(torch.from_numpy(srcs).cuda(), out)
        lanes = np.r_[np.arange(8), np.arange(1016, 1024), np.random.RandomState(1).choice(np.arange(8, 1016), 16,
                                                                                          replace=False)]
        ref = oracle.bfs_many(g, srcs[lanes])
        for j, c in enumerate(lanes):
            assert np.array_equal(out[int(c)].cpu().numpy(), ref[j]), (engine, int(c))
        del out


def test_closeness_rmat18_all_sources_sampled_targets(blest):
    g = gg.rmat(18, 16, seed=4)
    with blest.build_graph(g) as h:
        far, cc, reach = h.closeness()
    tg = gg.sources(g, 62, 9)
    tg = np.concatenate([tg, np.flatnonzero(np.diff(g.row_ptr) == 0)[:2]]).astype(np.int32)
    f_ref, r_ref = oracle.far_reach(g, tg)
    assert np.array_equal(far[tg], f_ref) and np.array_equal(reach[tg], r_ref)
    c_ref = oracle.closeness_from(f_ref, r_ref)
    nz = c_ref != 0
    assert np.all(cc[tg][~nz] == 0)
    assert np.all(np.abs(cc[tg][nz] - c_ref[nz]) <= 1e-12 * np.abs(c_ref[nz]))


def test_closeness_grid2048_two_batches_sampled_targets(blest):
    g = gg.grid(2048, 2048, 0.05, 0.001, seed=4)
    with blest.build_graph(g) as h:
        far, reach = h.closeness_range(0, 2048)
    tg = gg.sources(g, 32, 11)
    for t, d in zip(tg, oracle.bfs_many(g, tg)):
        d = d[:2048]
        assert far[t] == int(d[d >= 0].sum()) and reach[t] == int((d >= 0).sum())


def test_bfs_many_10000_ba_graphs_sampled(blest):
    b = gg.ba_batch(10000, 1000, 100000, 4, seed=3)
    rs = np.random.RandomState(0)
    srcs = np.array([rs.randint(0, int(b.vtx_off[i + 1] - b.vtx_off[i])) for i in range(b.g)], np.int32)
    with blest.build_many(b) as h:
        out = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device="cuda")
        h.bfs_many(srcs, out)
        got = out.cpu().numpy()
    sizes = np.diff(b.vtx_off)
    pick = np.concatenate([np.argsort(sizes)[-8:], np.argsort(sizes)[:8], rs.choice(b.g, 48, replace=False)])
    for i in pick:
        a, e = int(b.vtx_off[i]), int(b.vtx_off[i + 1])
        assert np.array_equal(got[a:e], oracle.bfs(b.graph(int(i)), int(srcs[i]))), int(i)


@pytest.mark.parametrize("family", ["rmat25", "ba16m_m8", "rgg16m"])
def test_held_out_families_sampled_sources(blest, family):
    if family == "rmat25":
        g = gg.rmat(25, 16, seed=25)
    elif family == "ba16m_m8":
        g = gg.ba(1 << 24, 8, seed=26)
    else:
        g = gg.rgg(1 << 24, 10.0, seed=27)
    with blest.build_graph(g) as h:
        _check_sources(blest, h, g, gg.sources(g, 64, 5)[:16])


def test_closeness_lattice2048_first_row_closed_form(blest):
    """Unperturbed 2048 x 2048 lattice, sources = row 0 (ids 0..2047, two
    batches of 1024): the distance sum to (r, c) is sum over c' of
    r + |c - c'| = 2048 r + c(c+1)/2 + (2047-c)(2048-c)/2, for every vertex."""
    R = C = 2048
    g = gg.lattice(R, C)
    with blest.build_graph(g) as h:
        far, reach = h.closeness_range(0, C)
    r, c = np.divmod(np.arange(R * C, dtype=np.int64), C)
    expect = C * r + c * (c + 1) // 2 + (C - 1 - c) * (C - c) // 2
    assert np.array_equal(far, expect)
    assert np.all(reach == C)
