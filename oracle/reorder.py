"""CPU oracle for the two vertex reorderings of §4.  TEST INFRASTRUCTURE ONLY.

Both return new_of_old: new_of_old[v] = position of original vertex v.

rcm: Cuthill-McKee (§4.2) -- repeatedly start from the unvisited vertex of
    smallest (degree, id), visit breadth-first, and append the unvisited
    neighbours of each dequeued vertex in ascending (degree, id) order; the
    whole visit order is then reversed.

jaccard_with_windows: Algorithm 1 (§4.1), one window at a time, each step in
    the paper's order: seed = highest-degree unassigned column of the window,
    R = its rows, inter[j] = |R & nbrs(j)| over the unassigned columns, Q =
    those with inter > 0; the remaining slots take the Q column maximising
    inter / (|R| + deg - inter) (or the highest-degree unassigned column when
    Q is empty), after which R and inter are updated with the new rows.
    Tie-breaks (the paper gives none): lowest column index; the ratio is
    compared exactly as integer cross-products.  The last, partial window
    runs ceil((w_e - w_s) / sigma) slice sets (the floor printed in
    Algorithm 1 would leave columns unassigned; read as a typo).
    nbrs(j) = out-neighbours of j (the nonzeros of column j of A); for the
    incremental update, the columns of row i are the in-neighbours of i,
    which equal the neighbours on an undirected graph.

symmetrized: a directed graph is reordered through its symmetrised pattern
    G + G^T (a reading: RCM is defined for symmetric patterns, and Algorithm
    1's incremental update assumes the in- and out-neighbours coincide); the
    orderings above then run on that graph unchanged.
"""
from __future__ import annotations

from collections import deque

import numpy as np


def rcm(g) -> np.ndarray:
    n = g.n
    rp, col = g.row_ptr, g.col
    deg = np.diff(rp)
    visited = np.zeros(n, bool)
    order = []
    starts = sorted(range(n), key=lambda v: (int(deg[v]), v))
    si = 0
    while len(order) < n:
        while visited[starts[si]]:
            si += 1
        s = starts[si]
        visited[s] = True
        q = deque([s])
        while q:
            v = q.popleft()
            order.append(v)
            nb = [int(w) for w in col[rp[v]:rp[v + 1]] if not visited[w]]
            nb.sort(key=lambda w: (int(deg[w]), w))
            for w in nb:
                visited[w] = True
                q.append(w)
    order.reverse()
    new_of_old = np.empty(n, np.int64)
    new_of_old[np.array(order, np.int64)] = np.arange(n)
    return new_of_old


def jaccard_with_windows(g, sigma: int = 8, W: int = 65536) -> np.ndarray:
    assert W % sigma == 0 and W > sigma
    n = g.n
    rp, col = g.row_ptr, g.col
    deg = np.diff(rp).astype(np.int64)
    nbrs = [col[rp[j]:rp[j + 1]] for j in range(n)]          # nbrs_A(j) and, undirected, nbrs_At(i)
    new_of_old = np.full(n, -1, np.int64)
    for w in range((n + W - 1) // W):
        ws, we = w * W, min(w * W + W, n)
        assigned = np.zeros(we - ws, bool)
        by_degree = sorted(range(ws, we), key=lambda j: (-int(deg[j]), j))
        ptr = 0

        def next_by_degree():
            nonlocal ptr
            while assigned[by_degree[ptr] - ws]:
                ptr += 1
            return by_degree[ptr]

        for s in range((we - ws + sigma - 1) // sigma):
            ss = ws + s * sigma
            se = min(ss + sigma, we)
            j = next_by_degree()
            assigned[j - ws] = True
            new_of_old[j] = ss
            R = set(int(i) for i in nbrs[j])
            inter = {}
            for i in R:
                for jj in nbrs[i]:
                    jj = int(jj)
                    if ws <= jj < we and not assigned[jj - ws]:
                        inter[jj] = inter.get(jj, 0) + 1
            Q = set(inter)
            for slot in range(ss + 1, se):
                if not Q:
                    j = next_by_degree()
                else:
                    best, bnum, bden = None, 0, 1
                    for jj in sorted(Q):
                        num = inter[jj]
                        den = len(R) + int(deg[jj]) - num
                        if best is None or num * bden > bnum * den:
                            best, bnum, bden = jj, num, den
                    j = best
                assigned[j - ws] = True
                Q.discard(j)
                new_of_old[j] = slot
                for i in nbrs[j]:
                    i = int(i)
                    if i in R:
                        continue
                    R.add(i)
                    for jj in nbrs[i]:
                        jj = int(jj)
                        if ws <= jj < we and not assigned[jj - ws]:
                            if inter.get(jj, 0) == 0:
                                Q.add(jj)
                            inter[jj] = inter.get(jj, 0) + 1
    assert np.all(new_of_old >= 0)
    return new_of_old


def jaccard_greedy_recompute(g, sigma: int = 8, W: int = 65536) -> np.ndarray:
    """The same greedy choice as jaccard_with_windows, but recomputing
    |R & nbrs(j)| from scratch at every step instead of updating it
    incrementally (a brute-force cross-check of the bookkeeping)."""
    n = g.n
    rp, col = g.row_ptr, g.col
    deg = np.diff(rp).astype(np.int64)
    nb = [set(int(x) for x in col[rp[j]:rp[j + 1]]) for j in range(n)]
    new_of_old = np.full(n, -1, np.int64)
    for w in range((n + W - 1) // W):
        ws, we = w * W, min(w * W + W, n)
        free = set(range(ws, we))

        def top_degree():
            return min(free, key=lambda j: (-int(deg[j]), j))

        for s in range((we - ws + sigma - 1) // sigma):
            ss = ws + s * sigma
            se = min(ss + sigma, we)
            j = top_degree()
            free.discard(j)
            new_of_old[j] = ss
            R = set(nb[j])
            for slot in range(ss + 1, se):
                cand = [(len(R & nb[c]), c) for c in sorted(free)]
                cand = [(x, c) for x, c in cand if x > 0]
                if not cand:
                    j = top_degree()
                else:
                    best = None
                    for x, c in cand:
                        den = len(R) + int(deg[c]) - x
                        if best is None or x * best[1] > best[0] * den:
                            best = (x, den, c)
                    j = best[2]
                free.discard(j)
                new_of_old[j] = slot
                R |= nb[j]
    return new_of_old


def bandwidth(g, new_of_old) -> int:
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    if len(src) == 0:
        return 0
    p = np.asarray(new_of_old)
    return int(np.abs(p[src] - p[g.col]).max())


def permute(g, new_of_old):
    """The graph relabelled by new_of_old (rows sorted)."""
    import graphgen as gg
    p = np.asarray(new_of_old, np.int64)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    out = gg.from_edges(g.n, p[src].astype(np.int32), p[g.col].astype(np.int32), symmetrize=False)
    out.directed = g.directed
    return out


class _Csr:
    """A plain CSR graph (n, row_ptr, col) for the oracle's own use."""

    def __init__(self, n, row_ptr, col):
        self.n, self.row_ptr, self.col, self.directed = n, row_ptr, col, False


def symmetrized(g):
    """G + G^T: every arc in both directions, duplicates and self loops
    dropped, rows sorted."""
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(g.row_ptr))
    dst = g.col.astype(np.int64)
    u = np.concatenate([src, dst])
    v = np.concatenate([dst, src])
    keep = u != v
    key = np.unique(u[keep] * n + v[keep])
    rows, cols = key // n, key % n
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return _Csr(n, np.cumsum(rp), cols.astype(np.int32))
