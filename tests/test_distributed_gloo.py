"""The source-range split of closeness across processes, on CPU: two gloo
ranks each sum the distances from their own sources (the oracle's serial
BFS stands in for the GPU batches) and one all-reduce completes far, reach
and cc, which must equal the single-process oracle exactly."""
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
