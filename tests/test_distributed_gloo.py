"""The source-range split of closeness across processes, on CPU: two gloo
ranks each sum the distances from their own sources (the oracle's serial
BFS stands in for the GPU batches) and one all-reduce completes far, reach
and cc, which must equal the single-process oracle exactly.  The resumable
run is tested the same way: a failure injected on the host part-way through,
then a rerun that must resume after the last saved chunk and end bit-exact."""
import os
import socket

import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _partial_oracle(g):
    def partial(first, count):
        far = np.zeros(g.n, np.int64)
        reach = np.zeros(g.n, np.int64)
        for s in range(first, first + count):
            d = oracle.bfs(g, s)
            ok = d >= 0
            far[ok] += d[ok]
            reach[ok] += 1
        return far, reach
    return partial


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2606_05081_gb300.distributed import closeness_allreduce
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = gg.disjoint_union(gg.rmat(10, seed=3), gg.path(700), gg.from_edges(5, [], [], True))
    far, reach, cc = closeness_allreduce(_partial_oracle(g), g.n, rank, world, dist)
    dist.destroy_process_group()
    q.put((rank, far, reach, cc))


def test_source_ranges_cover_in_whole_batches():
    from paper_2606_05081_gb300.distributed import source_ranges
    for n, w in [(1, 1), (1000, 2), (5000, 3), (262144, 8), (4194304, 7), (3000, 5)]:
        rs = source_ranges(n, w)
        assert len(rs) == w
        pos = 0
        for first, count in rs:
            assert first == pos and count >= 0
            pos += count
        assert pos == n
        assert all(f % 1024 == 0 for f, c in rs if c > 0)


def test_closeness_two_gloo_ranks_equal_single_process():
    # the package imports libblest; the reduction itself needs no GPU
    pytest.importorskip("paper_2606_05081_gb300")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=300) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = gg.disjoint_union(gg.rmat(10, seed=3), gg.path(700), gg.from_edges(5, [], [], True))
    far_r, reach_r, cc_r = oracle.closeness(g)
    for rank, far, reach, cc in res:
        assert np.array_equal(far, far_r) and np.array_equal(reach, reach_r), rank
        assert np.array_equal(cc, cc_r), rank


class _Crash(RuntimeError):
    pass


def _counting(partial, fail_after=None):
    """partial wrapped to record its calls and raise after `fail_after` of them."""
    calls = []

    def run(first, count):
        if fail_after is not None and len(calls) == fail_after:
            raise _Crash("injected failure")
        calls.append((first, count))
        return partial(first, count)
    return run, calls


def test_checkpointed_closeness_resumes_after_a_failure(tmp_path):
    from paper_2606_05081_gb300.distributed import closeness_checkpointed
    g = gg.disjoint_union(gg.rmat(9, seed=5), gg.path(300), gg.from_edges(3, [], [], True))
    far_r, reach_r, _ = oracle.closeness(g)
    path = str(tmp_path / "cc.npz")
    run, calls = _counting(_partial_oracle(g), fail_after=2)
    with pytest.raises(_Crash):
        closeness_checkpointed(run, g.n, path, chunk=100)
    assert calls == [(0, 100), (100, 100)]
    with np.load(path) as ck:
        assert int(ck["next"]) == 200
    # the rerun starts after the last completed chunk and ends bit-exact
    run2, calls2 = _counting(_partial_oracle(g))
    far, reach = closeness_checkpointed(run2, g.n, path, chunk=100)
    assert calls2[0] == (200, 100) and sum(c for _, c in calls2) == g.n - 200
    assert np.array_equal(far, far_r) and np.array_equal(reach, reach_r)
    # a finished checkpoint runs nothing more
    run3, calls3 = _counting(_partial_oracle(g))
    far3, reach3 = closeness_checkpointed(run3, g.n, path, chunk=100)
    assert calls3 == [] and np.array_equal(far3, far_r) and np.array_equal(reach3, reach_r)


def test_checkpointed_ranges_sum_to_the_whole_and_reject_foreign_checkpoints(tmp_path):
    from paper_2606_05081_gb300.distributed import closeness_checkpointed, source_ranges
    g = gg.rmat(10, seed=8)
    far_r, reach_r, _ = oracle.closeness(g)
    far = np.zeros(g.n, np.int64)
    reach = np.zeros(g.n, np.int64)
    for rank, (first, count) in enumerate(source_ranges(g.n, 3)):
        f, r = closeness_checkpointed(_partial_oracle(g), g.n, str(tmp_path / f"r{rank}.npz"), first, count,
                                      chunk=300)
        far += f
        reach += r
    assert np.array_equal(far, far_r) and np.array_equal(reach, reach_r)
    with pytest.raises(ValueError):   # rank 0's checkpoint, another range
        closeness_checkpointed(_partial_oracle(g), g.n, str(tmp_path / "r0.npz"), 1, 10)
    with pytest.raises(ValueError):
        closeness_checkpointed(_partial_oracle(g), g.n, str(tmp_path / "x.npz"), 0, g.n + 1)


def test_checkpoint_of_another_graph_with_the_same_n_is_refused(tmp_path):
    from paper_2606_05081_gb300.distributed import closeness_checkpointed, graph_fingerprint
    g1 = gg.rmat(9, seed=5)
    g2 = gg.rmat(9, seed=6)                # same vertex count, other arcs
    assert g1.n == g2.n
    fp1, fp2 = graph_fingerprint(g1.row_ptr, g1.col), graph_fingerprint(g2.row_ptr, g2.col)
    assert fp1 != fp2 and fp1 == graph_fingerprint(g1.row_ptr.copy(), g1.col.copy())
    path = str(tmp_path / "cc.npz")
    run, _ = _counting(_partial_oracle(g1), fail_after=1)
    with pytest.raises(_Crash):
        closeness_checkpointed(run, g1.n, path, chunk=100, fingerprint=fp1)
    with pytest.raises(ValueError):
        closeness_checkpointed(_partial_oracle(g2), g2.n, path, chunk=100, fingerprint=fp2)
    far, reach = closeness_checkpointed(_partial_oracle(g1), g1.n, path, chunk=100, fingerprint=fp1)
    far_r, reach_r, _ = oracle.closeness(g1)
    assert np.array_equal(far, far_r) and np.array_equal(reach, reach_r)


def test_reduction_runs_on_the_host_for_gloo_and_on_the_gpu_for_nccl():
    from paper_2606_05081_gb300.distributed import reduce_device

    class FakeDist:
        def __init__(self, backend):
            self.backend = backend

        def get_backend(self, group=None):
            return self.backend

    assert reduce_device(None).type == "cpu"
    assert reduce_device(FakeDist("gloo")).type == "cpu"
    if torch.cuda.is_available():
        assert reduce_device(FakeDist("nccl")).type == "cuda"


class _WallTimer:
    def start(self):
        import time
        self.t = time.perf_counter()

    def stop(self):
        import time
        return (time.perf_counter() - self.t) * 1e3


class _OracleHandle:
    """Stands in for a library handle: closeness_range from the oracle, and
    a record of the ranges it was asked for."""

    def __init__(self, g):
        self.partial = _partial_oracle(g)
        self.calls = []

    def closeness_range(self, first, count, far, reach):
        self.calls.append((first, count))
        f, r = self.partial(first, count)
        far[:] = f
        reach[:] = r


def _bench_split_worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = gg.rmat(11, seed=12)
    h = _OracleHandle(g)
    far = np.zeros(g.n, np.int64)
    reach = np.zeros(g.n, np.int64)
    ms, f, r, cc, rng = bench.closeness_split_run(h, g.n, rank, world, dist, far, reach, _WallTimer())
    dist.destroy_process_group()
    q.put((rank, h.calls, rng, f, r, cc, ms))


def test_bench_closeness_splits_sources_over_the_ranks():
    """The bench's closeness path runs only this rank's source range and
    all-reduces: two gloo ranks, each asked for its own half, end with the
    oracle's whole result."""
    pytest.importorskip("paper_2606_05081_gb300")
    from paper_2606_05081_gb300.distributed import source_ranges
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_bench_split_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted([q.get(timeout=300) for _ in ps], key=lambda x: x[0])
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = gg.rmat(11, seed=12)
    far_r, reach_r, cc_r = oracle.closeness(g)
    ranges = source_ranges(g.n, 2)
    for rank, calls, rng, f, r, cc, ms in res:
        assert calls == [ranges[rank]] and tuple(rng) == ranges[rank]
        assert np.array_equal(f, far_r) and np.array_equal(r, reach_r) and np.array_equal(cc, cc_r)
    assert res[0][6] == res[1][6]          # the max over ranks
