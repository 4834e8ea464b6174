"""GPU parity of multi-source BFS (Algorithm 5) and closeness (Eq. 6-7)
against the CPU oracle: levels and distance sums bit-exact, closeness values
within 1e-12 relative."""
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


MAKERS = {
    "rmat12": lambda: gg.rmat(12, seed=3),
    "grid_ragged": lambda: gg.grid(45, 61, seed=4),
    "er_directed": lambda: gg.er(3001, 12000, seed=5, directed=True),
    "union": lambda: gg.disjoint_union(gg.rmat(10, seed=6), gg.cycle(33), gg.from_edges(4, [], [], True)),
}


@pytest.mark.parametrize("tau", [128, 32])
@pytest.mark.parametrize("name", sorted(MAKERS))
@pytest.mark.parametrize("k", [1, 37, 64, 200, 256, 700, 1024])
def test_msbfs_levels(blest, name, k, tau):
    g = MAKERS[name]()
    rs = np.random.RandomState(k)
    srcs = rs.randint(0, g.n, size=k).astype(np.int32)   # duplicates allowed
    ref = oracle.bfs_many(g, srcs)
    with blest.build_graph(g, tau=tau) as h:
        got = h.msbfs(srcs)
        assert got.shape == ref.shape
        bad = np.argwhere(got != ref)
        assert len(bad) == 0, (name, k, bad[:5])


def test_msbfs_device_output(blest):
    g = gg.rmat(11, seed=8)
    srcs = gg.sources(g, 300, 4)
    ref = oracle.bfs_many(g, srcs)
    with blest.build_graph(g) as h:
        out = torch.empty((len(srcs), g.n), dtype=torch.int32, device="cuda")
        h.msbfs(torch.from_numpy(srcs).cuda(), out)
        assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("maker", [lambda: gg.rmat(11, seed=9), lambda: gg.grid(40, 70, seed=10),
                                   lambda: gg.disjoint_union(gg.rmat(9, seed=1), gg.path(50),
                                                             gg.from_edges(3, [], [], True)),
                                   lambda: gg.star(2500), lambda: gg.lattice(33, 65)])
@pytest.mark.parametrize("tau", [128, 32])
def test_closeness_all_sources(blest, maker, tau):
    g = maker()
    far_r, reach_r, cc_r = oracle.closeness(g)
    with blest.build_graph(g, tau=tau) as h:
        far, cc, reach = h.closeness()
    assert np.array_equal(far, far_r)
    assert np.array_equal(reach, reach_r)
    nz = cc_r != 0
    assert np.all(cc[~nz] == 0)
    assert np.all(np.abs(cc[nz] - cc_r[nz]) <= 1e-12 * np.abs(cc_r[nz]))


def test_closeness_lattice_closed_form(blest):
    R, C = 48, 37
    g = gg.lattice(R, C)
    r, c = np.divmod(np.arange(R * C), C)
    sr = np.abs(np.arange(R)[:, None] - np.arange(R)[None, :]).sum(1)
    sc = np.abs(np.arange(C)[:, None] - np.arange(C)[None, :]).sum(1)
    with blest.build_graph(g) as h:
        far, cc, reach = h.closeness()
    assert np.array_equal(far, C * sr[r] + R * sc[c])
    assert np.all(reach == R * C)


def test_closeness_ranges_add_up(blest):
    g = gg.rmat(12, seed=12)
    with blest.build_graph(g) as h:
        f_all, _, r_all = h.closeness()
        f1, r1 = h.closeness_range(0, 1500)
        f2, r2 = h.closeness_range(1500, g.n - 1500)
    assert np.array_equal(f1 + f2, f_all) and np.array_equal(r1 + r2, r_all)
    # sampled targets: sum over the range's sources of d(s, u) = BFS from u
    u = gg.sources(g, 5, 3)
    lv = oracle.bfs_many(g, u)
    for k, v in enumerate(u):
        d = lv[k][:1500]
        assert f1[v] == int(d[d >= 0].sum())
        assert r1[v] == int((d >= 0).sum())


def test_closeness_checkpointed_resumes_on_the_gpu(blest, tmp_path):
    """Chunks of 1500 sources (not a multiple of the 1024-lane batch), an
    injected host failure after the first chunk, then a resumed run: equal to
    the oracle's all-source sums."""
    from paper_2606_05081_gb300.distributed import closeness_checkpointed
    g = gg.disjoint_union(gg.rmat(12, seed=13), gg.path(500))
    far_r, reach_r, _ = oracle.closeness(g)
    path = str(tmp_path / "cc.npz")
    with blest.build_graph(g) as h:
        calls = []

        def failing(first, count):
            if calls:
                raise RuntimeError("injected failure")
            calls.append(first)
            return h.closeness_range(first, count)
        with pytest.raises(RuntimeError):
            closeness_checkpointed(failing, g.n, path, chunk=1500)
        far, reach = closeness_checkpointed(h.closeness_range, g.n, path, chunk=1500)
    assert np.array_equal(far, far_r) and np.array_equal(reach, reach_r)


def test_msbfs_rejects_bad_args(blest):
    g = gg.path(10)
    with blest.build_graph(g) as h:
        for bad in ([], [10], [-1]):
            with pytest.raises((blest.BlestError, ValueError)):
                h.msbfs(np.array(bad, np.int32))
        with pytest.raises(blest.BlestError):
            h.msbfs(np.zeros(1025, np.int32))
    gd = gg.er(50, 100, seed=1, directed=True)
    with blest.build_graph(gd) as h:
        with pytest.raises(blest.BlestError) as e:
            h.closeness()
        assert e.value.code == blest.ERR_UNSUPPORTED


# ------------------------------------------------ batched small graphs
@pytest.mark.parametrize("engine_tc", [0, 1])
def test_bfs_many_matches_oracle(blest, engine_tc):
    b = gg.ba_batch(60, 50, 5000, 4, seed=11)
    srcs = np.array([int(gg.sources(b.graph(i), 1, 100 + i)[0]) for i in range(b.g)], np.int32)
    with blest.build_many(b, engine_tc=engine_tc) as h:
        for rep in range(2):   # second call replays the captured CUDA graph
            got = h.bfs_many(srcs, total_n=int(b.vtx_off[-1]))
            for i in range(b.g):
                a, e = int(b.vtx_off[i]), int(b.vtx_off[i + 1])
                assert np.array_equal(got[a:e], oracle.bfs(b.graph(i), int(srcs[i]))), (rep, i)
        out = torch.empty(int(b.vtx_off[-1]), dtype=torch.int32, device="cuda")
        h.bfs_many(srcs[::-1].copy() % 50, out)
        got = out.cpu().numpy()
        s2 = srcs[::-1].copy() % 50
        for i in range(b.g):
            a, e = int(b.vtx_off[i]), int(b.vtx_off[i + 1])
            assert np.array_equal(got[a:e], oracle.bfs(b.graph(i), int(s2[i])))


def test_bfs_many_ragged_sizes_and_isolated(blest):
    # graphs whose sizes are not multiples of 8, one with an isolated source
    gs = [gg.path(13), gg.cycle(9), gg.disjoint_union(gg.star(21), gg.from_edges(2, [], [], True)), gg.rmat(8, seed=4)]
    vo = np.cumsum([0] + [g.n for g in gs]).astype(np.int64)
    eo = np.cumsum([0] + [g.nnz for g in gs]).astype(np.int64)
    rp = np.concatenate([g.row_ptr for g in gs]).astype(np.int64)
    col = np.concatenate([g.col for g in gs]).astype(np.int32)
    batch = gg.Batch(len(gs), vo, eo, rp, col)
    srcs = np.array([5, 0, 22, 7], np.int32)
    with blest.build_many(batch) as h:
        got = h.bfs_many(srcs, total_n=int(vo[-1]))
    for i, g in enumerate(gs):
        assert np.array_equal(got[vo[i]:vo[i + 1]], oracle.bfs(g, int(srcs[i])))


def _expected_counters(g, k_lanes, kappa, levels, bvss):
    """The multi-source work counters implied by the oracle's levels: per
    level l, the sets holding a vertex some lane reached at l - 1 are queued
    (their VSSs processed), the sets holding a target of an arc from such a
    vertex are dirty, and each (slice set, row) slot ORs one word per
    32-lane group that has a frontier lane among the slot's columns."""
    n = g.n
    kw = kappa // 32
    nv_of_set = np.diff(bvss["realPtrs"])
    src = np.repeat(np.arange(n), np.diff(g.row_ptr))
    dst = g.col.astype(np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    slot = (src // 8) * n + dst                    # one BVSS slot per (slice set, row)
    order = np.argsort(slot, kind="stable")
    src, dst, slot = src[order], dst[order], slot[order]
    starts = np.flatnonzero(np.r_[True, slot[1:] != slot[:-1]])
    lanes_pad = np.zeros((kappa, n), bool)
    vss = hitw = dirty = nlev = 0
    ell = 1
    while True:
        act = levels == ell - 1                    # k x n frontier of level ell
        av = act.any(axis=0)
        sets = np.unique(np.flatnonzero(av) // 8)
        q = int(nv_of_set[sets].sum()) if len(sets) else 0
        if q == 0:
            break
        nlev += 1
        vss += q
        m = av[src]
        dirty += len(np.unique(dst[m] // 8))
        lanes_pad[:] = False
        lanes_pad[:k_lanes] = act
        words = np.packbits(lanes_pad.reshape(kw, 32, n), axis=1, bitorder="little")   # kw x 4 x n bytes
        wv = np.ascontiguousarray(words.transpose(2, 0, 1)).reshape(n, kw * 4).view(np.uint32)   # n x kw
        per_arc = wv[src]                                                              # arcs x kw
        per_slot = np.bitwise_or.reduceat(per_arc, starts, axis=0)
        hitw += int((per_slot != 0).sum())
        ell += 1
    return {"levels": nlev, "vss": vss, "dirty_sets": dirty, "hit_words": hitw}


@pytest.mark.parametrize("name,k,tau", [("rmat12", 64, 128), ("grid_ragged", 200, 128), ("er_directed", 37, 32),
                                        ("union", 700, 32)])
def test_msbfs_work_counters_match_the_oracle_levels(blest, name, k, tau):
    g = MAKERS[name]()
    srcs = gg.sources(g, k, 11)
    ref = oracle.bfs_many(g, srcs)
    kappa = 64 if k <= 64 else (256 if k <= 256 else 1024)
    want = _expected_counters(g, len(srcs), kappa, ref, oracle.bvss(g, 8, tau))
    with blest.build_graph(g, tau=tau) as h:
        h.set_msbfs_direction(0)             # push every level: the counts of Algorithm 5
        assert np.array_equal(h.msbfs(srcs), ref)
        st = h.msbfs_stats()
    assert st["kappa"] == kappa and st["launches"] == 1 and st["pull_levels"] == 0
    for f in ("levels", "vss", "dirty_sets", "hit_words"):
        assert st[f] == want[f], (f, st[f], want[f])


@pytest.mark.parametrize("name", sorted(MAKERS))
@pytest.mark.parametrize("k", [1, 37, 64, 200, 256, 700, 1024])
def test_msbfs_levels_tensor_core_engine(blest, name, k):
    """Stage 1 on the tcgen05 tensor cores (0/1 bf16 MMA per 128-lane tile
    and 64 slots): levels bit-exact against the oracle for every batch width."""
    g = MAKERS[name]()
    rs = np.random.RandomState(1000 + k)
    srcs = rs.randint(0, g.n, size=k).astype(np.int32)
    ref = oracle.bfs_many(g, srcs)
    with blest.build_graph(g) as h:
        h.set_msbfs_engine(True)
        got = h.msbfs(srcs)
        bad = np.argwhere(got != ref)
        assert len(bad) == 0, (name, k, bad[:5])
        # twice in a row, and back on CUDA cores: the same levels
        assert np.array_equal(h.msbfs(srcs), ref)
        h.set_msbfs_engine(False)
        assert np.array_equal(h.msbfs(srcs), ref)


@pytest.mark.parametrize("name,k", [("rmat12", 64), ("grid_ragged", 200), ("union", 700)])
def test_tensor_core_engine_work_counters(blest, name, k):
    g = MAKERS[name]()
    srcs = gg.sources(g, k, 11)
    ref = oracle.bfs_many(g, srcs)
    kappa = 64 if k <= 64 else (256 if k <= 256 else 1024)
    want = _expected_counters(g, len(srcs), kappa, ref, oracle.bvss(g, 8, 128))
    with blest.build_graph(g) as h:
        h.set_msbfs_engine(True)
        h.set_msbfs_direction(0)
        assert np.array_equal(h.msbfs(srcs), ref)
        st = h.msbfs_stats()
    for f in ("levels", "vss", "dirty_sets", "hit_words"):
        assert st[f] == want[f], (f, st[f], want[f])


def test_tensor_core_closeness_and_layout_check(blest):
    g = gg.disjoint_union(gg.rmat(10, seed=9), gg.path(70), gg.from_edges(3, [], [], True))
    f_r, r_r, cc_r = oracle.closeness(g)
    with blest.build_graph(g) as h:
        h.set_msbfs_engine(True)
        far, cc, reach = h.closeness()
        assert np.array_equal(far, f_r) and np.array_equal(reach, r_r)
        assert np.allclose(cc, cc_r, rtol=1e-12, atol=0)
    with blest.build_graph(g, tau=32) as h:
        with pytest.raises(blest.BlestError) as e:
            h.set_msbfs_engine(True)
        assert e.value.code == blest.ERR_UNSUPPORTED


@pytest.mark.parametrize("reindex,tracking", [(0, 0), (1, 0), (0, 1)])
@pytest.mark.parametrize("name", sorted(MAKERS))
@pytest.mark.parametrize("tau", [128, 32])
def test_msbfs_ablation_variants_levels(blest, name, tau, reindex, tracking):
    """The ablation's multi-source variants -- without getVI reindexing and /
    or without activeSets / dirtySets tracking -- give the same levels and
    closeness sums as Algorithm 5 in full."""
    g = MAKERS[name]()
    srcs = np.random.RandomState(5).randint(0, g.n, size=300).astype(np.int32)
    ref = oracle.bfs_many(g, srcs)
    with blest.build_graph(g, tau=tau) as h:
        h.set_msbfs_variant(reindex, tracking)
        assert np.array_equal(h.msbfs(srcs), ref)
        assert np.array_equal(h.msbfs(srcs[:40]), ref[:40])
        if not g.directed:
            far, cc, reach = h.closeness()
            f_r, r_r, _ = oracle.closeness(g)
            assert np.array_equal(far, f_r) and np.array_equal(reach, r_r)
        with pytest.raises(blest.BlestError):
            h.set_msbfs_engine(True)        # the tensor-core engine runs Algorithm 5 in full only
        h.set_msbfs_variant(True, True)
        assert np.array_equal(h.msbfs(srcs[:40]), ref[:40])


@pytest.mark.parametrize("direction", [0, 1, 2])
@pytest.mark.parametrize("name", sorted(MAKERS))
@pytest.mark.parametrize("tau", [128, 32])
@pytest.mark.parametrize("k", [37, 300, 1024])
def test_msbfs_directions_levels(blest, name, tau, k, direction):
    """Push (Algorithm 5), pull on dense levels, and pull on every level give
    the same levels; on a graph with directed arcs pulling reads the
    in-neighbours."""
    g = MAKERS[name]()
    srcs = np.random.RandomState(k + 3).randint(0, g.n, size=k).astype(np.int32)
    ref = oracle.bfs_many(g, srcs)
    with blest.build_graph(g, tau=tau) as h:
        h.set_msbfs_direction(direction)
        assert np.array_equal(h.msbfs(srcs), ref)
        st = h.msbfs_stats()
        if direction == 2:
            assert st["pull_levels"] == st["levels"] and st["pull_arcs"] > 0
        if direction == 0:
            assert st["pull_levels"] == 0 and st["pull_arcs"] == 0


@pytest.mark.parametrize("direction", [1, 2])
def test_pulled_closeness_and_mixed_engines(blest, direction):
    g = gg.disjoint_union(gg.rmat(11, seed=19), gg.grid(30, 33, seed=2), gg.from_edges(3, [], [], True))
    f_r, r_r, cc_r = oracle.closeness(g)
    srcs = gg.sources(g, 700, 13)
    ref = oracle.bfs_many(g, srcs)
    with blest.build_graph(g) as h:
        h.set_msbfs_direction(direction)
        far, cc, reach = h.closeness()
        assert np.array_equal(far, f_r) and np.array_equal(reach, r_r)
        assert np.allclose(cc, cc_r, rtol=1e-12, atol=0)
        h.set_msbfs_engine(True)             # tensor-core push levels mixed with pulled ones
        assert np.array_equal(h.msbfs(srcs), ref)
        far2, _, reach2 = h.closeness()
        assert np.array_equal(far2, f_r) and np.array_equal(reach2, r_r)


@pytest.mark.parametrize("staged", [1, 0])
@pytest.mark.parametrize("reorder", [0, 1])
@pytest.mark.parametrize("k", [5, 300, 1024])
def test_msbfs_output_paths_deep_and_reordered(blest, staged, reorder, k):
    """Both ways of writing the source-major levels (staged bytes plus the
    closing transpose, or direct int32 stores), on a reordered graph (the
    transpose reads row new_of_old[v] for output column v) and on a path of
    700 vertices whose levels run past the 253 a staged byte holds (deeper
    lanes go straight to the output and the transpose must leave them)."""
    g = gg.disjoint_union(gg.path(700), gg.rmat(10, seed=12), gg.grid(13, 29, seed=13))
    rs = np.random.RandomState(100 + k)
    srcs = np.r_[[0, 699, 350], rs.randint(0, g.n, size=k - 3)].astype(np.int32)
    ref = oracle.bfs_many(g, srcs)
    assert ref.max() > 300
    with blest.build_graph(g, reorder=reorder) as h:
        h.set_msbfs_output(bool(staged))
        got = h.msbfs(srcs)
        bad = np.argwhere(got != ref)
        assert len(bad) == 0, (staged, reorder, k, bad[:5])
        out = torch.full((k, g.n), 7, dtype=torch.int32, device="cuda")   # every element must be written
        h.msbfs(torch.from_numpy(srcs).cuda(), out)
        assert np.array_equal(out.cpu().numpy(), ref)


def test_msbfs_output_switch_between_calls(blest):
    """Staged and direct output alternate on one handle, and a smaller batch
    after a larger one reuses the larger rows."""
    g = gg.rmat(12, seed=14)
    with blest.build_graph(g) as h:
        for staged, k in ((1, 1024), (0, 200), (1, 64), (1, 1000), (0, 1)):
            srcs = gg.sources(g, k, k)
            h.set_msbfs_output(bool(staged))
            assert np.array_equal(h.msbfs(srcs), oracle.bfs_many(g, srcs)), (staged, k)
