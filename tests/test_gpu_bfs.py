"""GPU parity of the single-source BFS path against the CPU oracle.

Every comparison is element by element and bit-exact: BFS levels, BVSS
arrays and per-level frontier counts are integers.  U_div is a float
statistic compared at 1e-12 relative (fp64 on both sides, different
summation order).
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


def _graphs():
    return {
        "rmat12": lambda: gg.rmat(12, seed=1),
        "rmat10_ef4": lambda: gg.rmat(10, edge_factor=4, seed=7),
        "grid_ragged": lambda: gg.grid(37, 53, seed=3),
        "ba": lambda: gg.ba(3001, 3, seed=4),
        "rgg": lambda: gg.rgg(4099, 8, seed=5),
        "er_directed": lambda: gg.er(2501, 9000, seed=6, directed=True),
        "star": lambda: gg.star(1500),
        "path": lambda: gg.path(1003),
        "union": lambda: gg.disjoint_union(gg.rmat(9, seed=2), gg.path(17), gg.from_edges(5, [], [], True)),
    }


GRAPHS = _graphs()
# (sigma, tau): the warp-wide VSS of each slice width, and the narrow sigma = 8 VSS
LAYOUTS = [(8, 128), (8, 32), (16, 64), (32, 32)]


@pytest.fixture(scope="module", params=[(g, s, t) for g in sorted(GRAPHS) for s, t in LAYOUTS],
                ids=lambda p: f"{p[0]}-s{p[1]}t{p[2]}")
def case(request, blest):
    name, sigma, tau = request.param
    g = GRAPHS[name]()
    h = blest.build_graph(g, sigma=sigma, tau=tau)
    yield name, g, h
    h.close()


def test_bvss_matches_oracle(case):
    name, g, h = case
    info = h.info()
    ref = oracle.bvss(g, info["sigma"], info["tau"])
    got = h.bvss()
    assert got["Nv"] == ref["Nv"] and got["Ns"] == ref["Ns"]
    assert np.array_equal(got["realPtrs"], ref["realPtrs"])
    assert np.array_equal(got["v2r"], ref["v2r"])
    assert np.array_equal(got["rowIds"], ref["rowIds"])
    assert np.array_equal(got["masks"], ref["masks"])
    assert info["nnz"] == g.nnz and info["num_slices"] == ref["num_slices"]
    u = oracle.update_divergence(ref)
    assert abs(info["update_divergence"] - u) <= 1e-12 * max(1.0, abs(u))


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_fixed_mode_levels(case, blest, mode):
    name, g, h = case
    h.set_policy(blest.POLICY_FIXED, mode)
    try:
        srcs = gg.sources(g, 6, 17)
        for s in srcs:
            assert np.array_equal(h.bfs(int(s)), oracle.bfs(g, int(s))), (name, mode, s)
    finally:
        h.set_policy(blest.POLICY_HEURISTIC)


def test_heuristic_and_random_schedules(case, blest):
    name, g, h = case
    srcs = gg.sources(g, 4, 23)
    refs = [oracle.bfs(g, int(s)) for s in srcs]
    for s, r in zip(srcs, refs):
        assert np.array_equal(h.bfs(int(s)), r)
    rs = np.random.RandomState(5)
    for trial in range(4):
        h.set_schedule(rs.randint(0, 5, size=rs.randint(1, 9)))
        h.set_policy(blest.POLICY_SCHEDULE)
        for s, r in zip(srcs, refs):
            assert np.array_equal(h.bfs(int(s)), r), (name, trial, s)
    h.set_policy(blest.POLICY_HEURISTIC)


@pytest.mark.parametrize("defer", [1, 0])
def test_deferred_queue_with_every_mode_transition(case, blest, defer):
    """Lazy and bottom-up levels that defer their VSS queue (counted, then
    written from the slice-set list by a top-down level that follows):
    levels are exact under schedules that cover every pair of modes, and
    the logged queue lengths equal those of the levels that write it."""
    name, g, h = case
    srcs = gg.sources(g, 3, 29)
    refs = [oracle.bfs(g, int(s)) for s in srcs]
    schedules = [[2, 0], [2, 2], [4, 0], [4, 2], [4, 4, 0], [2, 4, 1, 3, 4], [3, 0, 4, 3, 4, 2, 1]]
    try:
        for sched in schedules:
            h.set_schedule(sched)
            h.set_policy(blest.POLICY_SCHEDULE)
            logs = {}
            for d in (defer, 1 - defer):
                h.set_queue_deferral(d)
                for s, r in zip(srcs, refs):
                    assert np.array_equal(h.bfs(int(s)), r), (name, sched, d, int(s))
                logs[d] = [(x["level"], x["queue"], x["frontier"]) for x in h.level_log()]
            assert logs[0] == logs[1], (name, sched)
    finally:
        h.set_queue_deferral(-1)
        h.set_policy(blest.POLICY_HEURISTIC)


def test_device_output_and_level_log(case, blest):
    name, g, h = case
    s = int(gg.sources(g, 1, 31)[0])
    out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
    h.bfs(s, out)
    ref = oracle.bfs(g, s)
    assert np.array_equal(out.cpu().numpy(), ref)
    log = h.level_log()
    depth = int(ref.max())
    counts = np.bincount(ref[ref >= 0])
    deg = np.diff(g.row_ptr)
    info = h.info()
    sigma, tau = info["sigma"], info["tau"]
    b = oracle.bvss(g, sigma, tau)
    per_set = np.diff(b["realPtrs"])
    # one record per level whose input queue is non-empty: levels 1..depth,
    # plus the level that scans the deepest frontier when it owns any VSS
    last_q = int(per_set[np.unique(np.flatnonzero(ref == depth) // sigma)].sum())
    assert len(log) == depth + (1 if last_q > 0 else 0)
    visited = 0
    for k, rec in enumerate(log):
        assert rec["level"] == k + 1
        frontier = np.flatnonzero(ref == k)
        assert rec["frontier"] == counts[k]
        assert rec["frontier_edges"] == int(deg[frontier].sum())
        visited += counts[k]
        assert rec["unvisited"] == g.n - visited
        assert rec["queue"] == int(per_set[np.unique(frontier // sigma)].sum())
        assert rec["slots"] == rec["queue"] * tau
        assert 0 <= rec["mode"] < 5 and rec["t_ns"] >= 0
        assert 0 <= rec["t_stage1_ns"] <= rec["t_ns"]


def test_edge_cases(blest):
    # single vertex, no edges
    one = gg.from_edges(1, [], [], True)
    with blest.build(1, one.row_ptr, np.zeros(1, np.int32)) as h:
        assert h.bfs(0).tolist() == [0]
    # isolated source in a larger graph; n not a multiple of 8 or 32
    g = gg.disjoint_union(gg.cycle(45), gg.from_edges(3, [], [], True))
    with blest.build_graph(g) as h:
        lv = h.bfs(46)
        assert lv[46] == 0 and (lv >= 0).sum() == 1
        assert np.array_equal(h.bfs(3), oracle.bfs(g, 3))
        with pytest.raises(blest.BlestError) as e:
            h.bfs(48)
        assert e.value.code == blest.ERR_INVALID
        keep = np.full(g.n, 9, np.int32)
        with pytest.raises(blest.BlestError):
            h.bfs(-1, keep)
        assert np.all(keep == 9)


def test_malformed_csr_is_rejected(blest):
    rp = np.array([0, 2, 1, 3], np.int64)
    col = np.array([1, 2, 0], np.int32)
    with pytest.raises(blest.BlestError) as e:
        blest.build(3, rp, col)
    assert e.value.code == blest.ERR_INVALID
    rp = np.array([0, 1, 2, 3], np.int64)
    col = np.array([1, 2, 3], np.int32)  # 3 out of range
    with pytest.raises(blest.BlestError) as e:
        blest.build(3, rp, col)
    assert e.value.code == blest.ERR_INVALID


def test_duplicates_and_self_loops_change_nothing(blest):
    g = gg.rmat(10, seed=11)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    # add every arc twice plus a self loop on each vertex, unsorted rows
    u = np.concatenate([src, src, np.arange(g.n)]).astype(np.int32)
    v = np.concatenate([g.col, g.col, np.arange(g.n)]).astype(np.int32)
    order = np.random.RandomState(0).permutation(len(u))
    u, v = u[order], v[order]
    rp = np.zeros(g.n + 1, np.int64)
    np.add.at(rp, u + 1, 1)
    rp = np.cumsum(rp)
    col = v[np.argsort(u, kind="stable")]
    with blest.build(g.n, rp, col.astype(np.int32)) as h:
        assert h.info()["nnz"] == g.nnz
        ref = oracle.bvss(g, 8)
        got = h.bvss()
        assert np.array_equal(got["masks"], ref["masks"]) and np.array_equal(got["rowIds"], ref["rowIds"])
        for s in gg.sources(g, 3, 2):
            assert np.array_equal(h.bfs(int(s)), oracle.bfs(g, int(s)))


def test_barrier_timeout_returns_status_and_context_survives(blest):
    assert blest.selftest_barrier_timeout(20) == blest.ERR_TIMEOUT
    g = gg.path(100)
    with blest.build_graph(g) as h:
        assert np.array_equal(h.bfs(0), np.arange(100))


def test_rmat16_64_sources_bit_exact(blest):
    """Scale-16 RMAT, edge factor 16, no reordering, 64 seeded sources of
    nonzero degree, heuristic policy (the small single-source workload)."""
    g = gg.rmat(16, seed=1)
    srcs = gg.sources(g, 64, 1)
    ref = oracle.bfs_many(g, srcs)
    with blest.build_graph(g) as h:
        info = h.info()
        assert info["lazy"] == 0  # U_div below 25,000 -> Algorithm 2
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for k, s in enumerate(srcs):
            h.bfs(int(s), out)
            assert np.array_equal(out.cpu().numpy(), ref[k]), k


def test_layout_options_are_checked(blest):
    g = gg.rmat(9, seed=3)
    for sigma, tau in [(8, 64), (16, 32), (16, 128), (32, 64), (12, 0)]:
        with pytest.raises(blest.BlestError) as e:
            blest.build_graph(g, sigma=sigma, tau=tau)
        assert e.value.code == blest.ERR_INVALID, (sigma, tau)
    # the b1 MMA hit test needs the Fig. 3 layout
    with pytest.raises(blest.BlestError) as e:
        blest.build_graph(g, sigma=8, tau=32, engine_tc=1)
    assert e.value.code == blest.ERR_UNSUPPORTED
    with blest.build_graph(g, sigma=16) as h:
        assert h.info()["tau"] == 64
        with pytest.raises(blest.BlestError) as e:
            h.set_engine(True)
        assert e.value.code == blest.ERR_UNSUPPORTED
        # a fixed tensor-core mode runs its CUDA-core twin and the log says so
        h.set_policy(blest.POLICY_FIXED, blest.MODE_PUSH_LAZY_TC)
        s = int(gg.sources(g, 1, 3)[0])
        assert np.array_equal(h.bfs(s), oracle.bfs(g, s))
        assert {r["mode"] for r in h.level_log()} == {blest.MODE_PUSH_LAZY_CC}
        # multi-source BFS and closeness group the 8 vertices of a slice set
        with pytest.raises(blest.BlestError) as e:
            h.msbfs(np.array([s], np.int32))
        assert e.value.code == blest.ERR_UNSUPPORTED


@pytest.mark.parametrize("sigma,tau", LAYOUTS)
def test_reordered_layouts_bit_exact(blest, sigma, tau):
    """RCM and JaccardWithWindows (slice sets of sigma columns) under every
    layout: levels equal the oracle's on the original graph."""
    for g, reorder in [(gg.grid(61, 67, 0.05, 0.001, seed=8), blest.REORDER_RCM),
                       (gg.rmat(12, seed=9), blest.REORDER_JACCARD)]:
        with blest.build_graph(g, sigma=sigma, tau=tau, reorder=reorder, jaccard_window=1024) as h:
            assert h.info()["reorder"] == reorder
            for s in gg.sources(g, 3, 4):
                for mode in (0, 2, 4):
                    h.set_policy(blest.POLICY_FIXED, mode)
                    assert np.array_equal(h.bfs(int(s)), oracle.bfs(g, int(s))), (reorder, mode, s)


@pytest.mark.parametrize("tau", [128, 32])
def test_hub_slice_sets_and_queue_counts(blest, tau):
    """Hubs whose slice sets span hundreds of VSSs (ranges the whole warp
    writes): levels exact in eager and lazy modes, and the logged queue
    length of every level equals the VSS count of the slice sets holding the
    previous level's vertices."""
    stars = gg.disjoint_union(gg.star(20000), gg.star(9000), gg.rmat(13, seed=3))
    ref_b = oracle.bvss(stars, 8, tau)
    nv_of_set = np.diff(ref_b["realPtrs"])
    assert nv_of_set.max() >= 64 * (128 // tau)
    with blest.build_graph(stars, tau=tau) as h:
        for mode in [0, 2, 4, 1 if tau == 128 else 0]:
            h.set_policy(blest.POLICY_FIXED, mode)
            for s in [0, 20000, 29000, 29001 + 17]:
                lv = h.bfs(int(s))
                want = oracle.bfs(stars, int(s))
                assert np.array_equal(lv, want), (tau, mode, s)
                for rec in h.level_log():
                    prev = np.flatnonzero(want == rec["level"] - 1)
                    assert rec["queue"] == int(nv_of_set[np.unique(prev // 8)].sum()), (tau, mode, s, rec)
        h.set_policy(blest.POLICY_HEURISTIC)


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_sixteen_mma_layout_levels(blest, name):
    """Tensor-core levels with one slice per fragment row (16 MMAs per VSS,
    the layout the ablation measures Fig. 3's against): levels exact in the
    eager and lazy tensor-core modes and under the paper's rule."""
    g = GRAPHS[name]()
    with blest.build_graph(g) as h:
        h.set_engine(2)
        assert h.info()["engine_tc"] == 2
        srcs = gg.sources(g, 4, 29)
        for pol, mode in [(blest.POLICY_FIXED, 1), (blest.POLICY_FIXED, 3), (blest.POLICY_HEURISTIC, 0)]:
            h.set_policy(pol, mode)
            for s in srcs:
                assert np.array_equal(h.bfs(int(s)), oracle.bfs(g, int(s))), (name, pol, mode, s)
    with blest.build_graph(g, tau=32) as h:
        with pytest.raises(blest.BlestError):
            h.set_engine(2)


@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_pinned_and_pageable_host_output(blest, reorder):
    """Page-locked host buffers, 16-byte aligned or not, and a pageable one
    receive the levels of plain and reordered graphs, every element
    written."""
    g = gg.disjoint_union(gg.rmat(12, seed=41), gg.grid(17, 23, seed=42), gg.from_edges(5, [], [], True))
    srcs = gg.sources(g, 6, 43)
    refs = oracle.bfs_many(g, srcs)
    with blest.build_graph(g, reorder=reorder) as h:
        for off in (0, 1):   # 16-byte aligned, then not
            base = torch.full((g.n + 1,), 7, dtype=torch.int32).pin_memory()
            host = base.numpy()[off:off + g.n]
            for s, ref in zip(srcs, refs):
                h.bfs(int(s), host)
                assert np.array_equal(host, ref), (reorder, off, int(s))
        plain = np.full(g.n, 7, np.int32)
        h.bfs(int(srcs[0]), plain)
        assert np.array_equal(plain, refs[0])
