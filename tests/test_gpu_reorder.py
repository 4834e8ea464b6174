"""GPU reorderings (§4) against the CPU oracle: the permutation itself is
bit-exact (RCM and JaccardWithWindows use the same tie-breaks on both
sides), the BVSS of the reordered graph matches the oracle's BVSS of the
relabelled graph, and BFS / MS-BFS / closeness results come back in the
caller's original ids."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import reorder

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def blest():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2606_05081_gb300 as b
    return b


def _scrambled_lattice(R, C, seed):
    return reorder.permute(gg.lattice(R, C), np.random.RandomState(seed).permutation(R * C))


RCM_GRAPHS = {
    "grid": lambda: gg.grid(33, 47, seed=3),
    "scrambled_lattice": lambda: _scrambled_lattice(40, 60, 1),
    "union_isolated": lambda: gg.disjoint_union(gg.path(7), gg.from_edges(3, [], [], True), gg.cycle(11),
                                                gg.rmat(8, seed=2)),
    "star_big_level": lambda: gg.star(5000),
    "rmat12": lambda: gg.rmat(12, seed=5),
    "ba": lambda: gg.ba(4000, 3, seed=6),
}


@pytest.mark.parametrize("name", sorted(RCM_GRAPHS))
def test_rcm_permutation_matches_oracle(blest, name):
    g = RCM_GRAPHS[name]()
    with blest.build_graph(g, reorder=blest.REORDER_RCM) as h:
        assert h.info()["reorder"] == blest.REORDER_RCM
        p = h.perm()
    assert np.array_equal(p, reorder.rcm(g))


JAC_GRAPHS = {
    "rmat10_w64": (lambda: gg.rmat(10, seed=1), 64),
    "rmat11_w512": (lambda: gg.rmat(11, seed=2), 512),
    "ba_w96": (lambda: gg.ba(2000, 4, seed=3), 96),
    "grid_w80": (lambda: gg.grid(20, 30, seed=4), 80),
    "rmat12_w65536": (lambda: gg.rmat(12, seed=5), 65536),
    "star_w32": (lambda: gg.star(300), 32),
}


@pytest.mark.parametrize("name", sorted(JAC_GRAPHS))
def test_jaccard_permutation_matches_oracle(blest, name):
    mk, W = JAC_GRAPHS[name]
    g = mk()
    with blest.build_graph(g, reorder=blest.REORDER_JACCARD, jaccard_window=W) as h:
        assert h.info()["reorder"] == blest.REORDER_JACCARD
        p = h.perm()
    assert np.array_equal(p, reorder.jaccard_with_windows(g, 8, W))


@pytest.mark.parametrize("which", ["rcm", "jaccard"])
def test_reordered_bvss_and_levels(blest, which):
    g = gg.rmat(12, seed=9) if which == "jaccard" else gg.grid(30, 41, seed=8)
    opt = dict(reorder=blest.REORDER_RCM) if which == "rcm" else dict(reorder=blest.REORDER_JACCARD,
                                                                      jaccard_window=1024)
    with blest.build_graph(g, **opt) as h:
        p = h.perm()
        ref_b = oracle.bvss(reorder.permute(g, p), 8)
        got_b = h.bvss()
        assert np.array_equal(got_b["rowIds"], ref_b["rowIds"])
        assert np.array_equal(got_b["masks"], ref_b["masks"])
        srcs = gg.sources(g, 5, 3)
        for mode in range(5):
            h.set_policy(blest.POLICY_FIXED, mode)
            for s in srcs:
                assert np.array_equal(h.bfs(int(s)), oracle.bfs(g, int(s))), (mode, s)
        h.set_policy(blest.POLICY_HEURISTIC)
        ms = h.msbfs(srcs)
        assert np.array_equal(ms, oracle.bfs_many(g, srcs))
        far, cc, reach = h.closeness()
        f_r, r_r, _ = oracle.closeness(g)
        assert np.array_equal(far, f_r) and np.array_equal(reach, r_r)


def test_auto_reorder_classifies(blest):
    with blest.build_graph(gg.rmat(12, seed=1), reorder=blest.REORDER_AUTO, jaccard_window=1024) as h:
        assert h.info()["reorder"] == blest.REORDER_JACCARD      # scale-free-like degrees
    with blest.build_graph(gg.grid(40, 40, seed=2), reorder=blest.REORDER_AUTO) as h:
        assert h.info()["reorder"] == blest.REORDER_RCM


@pytest.mark.parametrize("which", ["rcm", "jaccard"])
def test_directed_graph_reorders_through_its_symmetrised_pattern(blest, which):
    g = gg.er(3000, 9000, seed=1, directed=True)
    if which == "rcm":
        opt, want = dict(reorder=blest.REORDER_RCM), reorder.rcm(reorder.symmetrized(g))
    else:
        opt = dict(reorder=blest.REORDER_JACCARD, jaccard_window=256)
        want = reorder.jaccard_with_windows(reorder.symmetrized(g), 8, 256)
    with blest.build_graph(g, **opt) as h:
        assert np.array_equal(h.perm(), want)
        srcs = gg.sources(g, 4, 2)
        for mode in range(5):
            h.set_policy(blest.POLICY_FIXED, mode)
            for s in srcs:
                assert np.array_equal(h.bfs(int(s)), oracle.bfs(g, int(s))), (mode, s)
        h.set_policy(blest.POLICY_HEURISTIC)
        assert np.array_equal(h.msbfs(srcs), oracle.bfs_many(g, srcs))


def _degree_sequences():
    """Hand-built sequences (the oracle's pins) and graph families."""
    from oracle import classify
    rng = np.random.default_rng(3)
    seqs = {
        "regular4": (np.full(1000, 4), None),
        "concentrated": (np.array([100] * 2 + [10] * 18 + [1] * 180), None),
        "powerlaw_only": (np.array([4] * 1_000_000 + sum(([k] * int(1e6 * k ** -3.0) for k in range(5, 61)), [])),
                          None),
        "steep": (np.array(sum(([k] * int(1e9 * k ** -6.0) for k in range(5, 12)), [])), None),
        "noisy": (np.array(sum(([k] * int(rng.integers(1, 50)) for k in range(5, 400)), [])), None),
        "one_point": (np.array([7] * 9), None),
        "in_star": (np.r_[0, np.ones(499, np.int64)], np.r_[499, np.zeros(499, np.int64)]),
    }
    for name, g in [("lattice", gg.lattice(64, 64)), ("grid", gg.grid(128, 128, 0.05, 0.001, seed=1)),
                    ("star", gg.star(300)), ("rmat14", gg.rmat(14, seed=1)), ("ba", gg.ba(1 << 15, 4, seed=2)),
                    ("er_directed", gg.er(5000, 40000, seed=3, directed=True))]:
        o, i = classify.degrees(g)
        seqs[name] = (o, i if g.directed else None)
    return seqs


def test_scale_free_test_matches_oracle(blest):
    from oracle import classify
    for name, (o, i) in _degree_sequences().items():
        got = blest.scale_free_test(o, i)
        want = classify.scale_free_like(o, i)
        assert got["scale_free"] == want["scale_free"], name
        for side in ("out", "in"):
            g_, w_ = got[side], want[side]
            assert g_["top1"] == w_["top1"] and g_["top10"] == w_["top10"], (name, side)   # exact integer sums
            assert g_["points"] == w_["points"], (name, side)
            for f in ("gamma", "r2"):
                if np.isnan(w_[f]):
                    assert np.isnan(g_[f]), (name, side, f)
                else:
                    assert g_[f] == pytest.approx(w_[f], rel=1e-9, abs=1e-12), (name, side, f)
            for f in ("concentrated", "powerlaw", "heavy"):
                assert bool(g_[f]) == w_[f], (name, side, f)


def test_scale_free_test_takes_device_arrays_and_rejects_negative_degrees(blest):
    from oracle import classify
    o, _ = classify.degrees(gg.rmat(12, seed=2))
    got = blest.scale_free_test(torch.from_numpy(o).cuda())
    assert got["scale_free"] == classify.scale_free_like(o)["scale_free"]
    with pytest.raises(blest.BlestError) as e:
        blest.scale_free_test(np.array([3, -1, 2]))
    assert e.value.code == blest.ERR_INVALID


def test_auto_reorder_follows_the_oracle_decision(blest):
    from oracle import classify
    for g in [gg.rmat(12, seed=1), gg.grid(40, 40, seed=2), gg.ba(3000, 3, seed=4), gg.lattice(30, 30),
              gg.er(3000, 9000, seed=5, directed=True)]:
        want = classify.scale_free_like(*classify.degrees(g)) if g.directed else \
            classify.scale_free_like(classify.degrees(g)[0])
        with blest.build_graph(g, reorder=blest.REORDER_AUTO, jaccard_window=1024) as h:
            assert h.info()["reorder"] == (blest.REORDER_JACCARD if want["scale_free"] else blest.REORDER_RCM)
