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


def test_reorder_directed_is_unsupported(blest):
    g = gg.er(100, 300, seed=1, directed=True)
    with pytest.raises(blest.BlestError) as e:
        blest.build_graph(g, reorder=blest.REORDER_RCM)
    assert e.value.code == blest.ERR_UNSUPPORTED
