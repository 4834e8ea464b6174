"""The allocation-free BFS entry point (blest_bfs_noalloc), checked against
the CPU oracle and against the regular entry point (blest_bfs).

blest_bfs_noalloc exists for callers that cannot call cudaMalloc -- code
whose device memory is all owned by another allocator, or latency-critical
paths that must not take cudaMalloc's implicit synchronisation.  It keeps
its scratch in a static device array shared by every call, so this file
checks two calls in a row (the second must not see stale state from the
first), a reordered graph (ids in the reordered numbering), and that views
beyond the array's size limit or of another BVSS layout are refused.  It is
named to be collected last: if it fails, every other test has already run.
"""
import ctypes

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


def _device_view(blest, h, deg, engine_tc):
    """A view of the handle's BVSS copied into caller-owned device buffers;
    deg is the out-degree array in the BVSS's (possibly reordered) ids."""
    info = h.info()
    nv, ns = info["num_vss"], info["num_slice_sets"]
    tau = info["tau"]
    dev = torch.device("cuda")
    bufs = dict(rows=torch.empty(max(nv, 1) * tau, dtype=torch.int32, device=dev),
                masks=torch.empty(max(nv, 1) * tau // 4, dtype=torch.int32, device=dev),
                real=torch.empty(ns + 1, dtype=torch.int32, device=dev),
                v2r=torch.empty(max(nv, 1), dtype=torch.int32, device=dev),
                deg=torch.from_numpy(np.ascontiguousarray(deg, dtype=np.int32)).to(dev))
    rc = blest._lib.blest_get_bvss(h._h, bufs["rows"].data_ptr(), bufs["masks"].data_ptr(),
                                   bufs["real"].data_ptr(), bufs["v2r"].data_ptr())
    assert rc == blest.OK
    view = blest.BvssView(n=info["n"], num_slice_sets=ns, num_vss=nv, row_ids=bufs["rows"].data_ptr(),
                          masks=bufs["masks"].data_ptr(), real_ptrs=bufs["real"].data_ptr(),
                          virtual_to_real=bufs["v2r"].data_ptr(), out_degree=bufs["deg"].data_ptr(),
                          engine_tc=engine_tc, sigma=info["sigma"], tau=tau)
    return view, bufs


@pytest.mark.parametrize("engine_tc", [1, 0])
def test_noalloc_matches_oracle_and_regular_entry_point_on_two_calls(blest, engine_tc):
    g = gg.rmat(15, seed=21)
    srcs = gg.sources(g, 2, 5)
    with blest.build_graph(g) as h:
        view, bufs = _device_view(blest, h, np.diff(g.row_ptr), engine_tc)
        torch.cuda.synchronize()
        for s in srcs:                      # two calls in a row, different sources
            want = oracle.bfs(g, int(s))
            out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
            blest.bfs_noalloc(view, int(s), out)
            got = out.cpu().numpy()
            assert np.array_equal(got, want)
            assert np.array_equal(got, h.bfs(int(s)))     # the existing entry point
        # and the first source again after the second: no stale state
        out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        blest.bfs_noalloc(view, int(srcs[0]), out)
        assert np.array_equal(out.cpu().numpy(), oracle.bfs(g, int(srcs[0])))


def test_noalloc_on_a_reordered_graph_works_in_reordered_ids(blest):
    g = gg.grid(48, 40, 0.05, 0.01, seed=3)
    srcs = gg.sources(g, 2, 9)
    with blest.build_graph(g, reorder=blest.REORDER_RCM) as h:
        perm = h.perm()                     # new_of_old
        assert not np.array_equal(perm, np.arange(g.n))
        deg_new = np.empty(g.n, np.int64)
        deg_new[perm] = np.diff(g.row_ptr)
        view, bufs = _device_view(blest, h, deg_new, 0)
        for s in srcs:
            out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
            blest.bfs_noalloc(view, int(perm[s]), out)
            got_new = out.cpu().numpy()
            assert np.array_equal(got_new[perm], oracle.bfs(g, int(s)))


def test_noalloc_refuses_views_it_cannot_run(blest):
    g = gg.path(64)
    with blest.build_graph(g) as h:
        view, bufs = _device_view(blest, h, np.diff(g.row_ptr), 1)
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        big = blest.BvssView.from_buffer_copy(view)
        big.n = (1 << 20) + 8
        big.num_slice_sets = (big.n + 7) // 8
        rc = blest._lib.blest_bfs_noalloc(ctypes.byref(big), 0, out.data_ptr(), None)
        assert rc == blest.ERR_UNSUPPORTED
        big = blest.BvssView.from_buffer_copy(view)
        big.num_vss = (1 << 17) + 1
        rc = blest._lib.blest_bfs_noalloc(ctypes.byref(big), 0, out.data_ptr(), None)
        assert rc == blest.ERR_UNSUPPORTED
        host = np.empty(g.n, np.int32)     # levels must be device memory
        rc = blest._lib.blest_bfs_noalloc(ctypes.byref(view), 0, host.ctypes.data, None)
        assert rc == blest.ERR_INVALID
    # a BVSS of the narrow tau = 32 layout (the autotuner's pick on grids)
    with blest.build_graph(g, tau=32) as h:
        view, bufs = _device_view(blest, h, np.diff(g.row_ptr), 0)
        assert view.tau == 32
        out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        rc = blest._lib.blest_bfs_noalloc(ctypes.byref(view), 0, out.data_ptr(), None)
        assert rc == blest.ERR_UNSUPPORTED
        assert int(out[0].item()) == 7       # refused before any launch
