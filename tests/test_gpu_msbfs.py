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
