"""Seeded synthetic graph inputs shared by the CPU oracle and the GPU path.

This module only *produces inputs* (CSR graphs and source lists); it holds
none of the BFS arithmetic.  The generators live in ``graphgen.c`` (compiled
on first use with the host gcc, no x86/Arm specific flags) and are
deterministic functions of their seed on any host and thread count.

Workloads (shapes and distributions of the paper's evaluation graphs, §7,
stood in for by synthetic families):
  * RMAT (Graph500 quadrant probabilities a=0.57, b=0.19, c=0.19) stands in
    for the Kronecker / social graphs (GAP-kron, GAP-urand, com-Friendster).
  * a 2D grid with edge deletions and random shortcuts stands in for the
    road networks (GAP-road, europe_osm).
  * Barabasi-Albert and 2D random geometric graphs stand in for the
    preferential-attachment and rgg_n_2_24 families.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_graphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into an in-tree shared library (idempotent)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32, u64, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
            lib.gg_rmat.restype = P
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int, dbl, dbl, dbl, u64, ctypes.c_int, ctypes.c_int]
            lib.gg_grid.restype = P
            lib.gg_grid.argtypes = [ctypes.c_int, ctypes.c_int, dbl, dbl, u64, ctypes.c_int]
            lib.gg_ba.restype = P
            lib.gg_ba.argtypes = [i64, ctypes.c_int, u64, ctypes.c_int]
            lib.gg_rgg.restype = P
            lib.gg_rgg.argtypes = [i64, dbl, u64, ctypes.c_int]
            lib.gg_er.restype = P
            lib.gg_er.argtypes = [i64, i64, u64, ctypes.c_int, ctypes.c_int]
            lib.gg_from_edges.restype = P
            lib.gg_from_edges.argtypes = [i64, i64, P, P, ctypes.c_int, ctypes.c_int]
            lib.gg_free.argtypes = [P]
            lib.gg_n.restype = i64
            lib.gg_n.argtypes = [P]
            lib.gg_nnz.restype = i64
            lib.gg_nnz.argtypes = [P]
            lib.gg_copy.argtypes = [P, P, P]
            lib.gg_sources.restype = ctypes.c_int
            lib.gg_sources.argtypes = [P, i64, ctypes.c_int, u64, P]
            lib.gg_rng.restype = u64
            lib.gg_rng.argtypes = [u64, u64, u64]
            lib.gg_ba_batch.restype = P
            lib.gg_ba_batch.argtypes = [i32, i64, i64, ctypes.c_int, u64, ctypes.c_int]
            lib.gg_batch_free.argtypes = [P]
            lib.gg_batch_g.restype = i32
            lib.gg_batch_g.argtypes = [P]
            lib.gg_batch_total_n.restype = i64
            lib.gg_batch_total_n.argtypes = [P]
            lib.gg_batch_total_nnz.restype = i64
            lib.gg_batch_total_nnz.argtypes = [P]
            lib.gg_batch_copy.argtypes = [P, P, P, P, P]
            _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


@dataclass
class Graph:
    """CSR graph: row v lists the out-neighbours of v (sorted, no duplicates,
    no self loops).  ``directed=False`` means the CSR is symmetric."""
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[nnz]
    directed: bool = False
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


@dataclass
class Batch:
    """Many small graphs concatenated: graph i owns vertices
    [vtx_off[i], vtx_off[i+1]) (local ids 0..n_i-1) and arcs
    [edge_off[i], edge_off[i+1]); its local CSR row pointer is
    row_ptr[vtx_off[i] + i : vtx_off[i+1] + i + 1] (relative to edge_off[i])."""
    g: int
    vtx_off: np.ndarray
    edge_off: np.ndarray
    row_ptr: np.ndarray
    col: np.ndarray

    def graph(self, i: int) -> Graph:
        a, b = int(self.vtx_off[i]), int(self.vtx_off[i + 1])
        rp = self.row_ptr[a + i: b + i + 1].copy()
        e0, e1 = int(self.edge_off[i]), int(self.edge_off[i + 1])
        return Graph(b - a, rp, self.col[e0:e1].copy(), False, f"batch[{i}]")


def _take(ptr, name: str, directed: bool = False) -> Graph:
    lib = _load()
    if not ptr:
        raise MemoryError(f"graph generator {name} failed")
    try:
        n, nnz = lib.gg_n(ptr), lib.gg_nnz(ptr)
        rp = np.empty(n + 1, dtype=np.int64)
        col = np.empty(max(nnz, 1), dtype=np.int32)
        lib.gg_copy(ptr, rp.ctypes.data, col.ctypes.data)
        return Graph(int(n), rp, col[:nnz], directed, name)
    finally:
        lib.gg_free(ptr)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, scramble: bool = True) -> Graph:
    """Undirected RMAT graph with n = 2^scale and edge_factor*n edge samples."""
    lib = _load()
    return _take(lib.gg_rmat(scale, edge_factor, a, b, c, seed, int(scramble), _threads()),
                 f"rmat{scale}_ef{edge_factor}")


def grid(rows: int, cols: int, delete_frac: float = 0.05, shortcut_frac: float = 0.001,
         seed: int = 2) -> Graph:
    """Road-like grid: 4-neighbour lattice, delete_frac of edges removed,
    floor(shortcut_frac * lattice edges) uniform random shortcuts added."""
    lib = _load()
    return _take(lib.gg_grid(rows, cols, delete_frac, shortcut_frac, seed, _threads()),
                 f"grid{rows}x{cols}")


def ba(n: int, m: int, seed: int = 5) -> Graph:
    lib = _load()
    return _take(lib.gg_ba(n, m, seed, _threads()), f"ba{n}_m{m}")


def rgg(n: int, avg_degree: float = 10.0, seed: int = 5) -> Graph:
    lib = _load()
    return _take(lib.gg_rgg(n, avg_degree, seed, _threads()), f"rgg{n}")


def er(n: int, m: int, seed: int = 9, directed: bool = False) -> Graph:
    lib = _load()
    return _take(lib.gg_er(n, m, seed, int(directed), _threads()), f"er{n}_{m}", directed)


def from_edges(n: int, u, v, symmetrize: bool = True, name: str = "edges") -> Graph:
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    assert u.shape == v.shape
    return _take(lib.gg_from_edges(n, len(u), u.ctypes.data, v.ctypes.data, int(symmetrize), _threads()),
                 name, directed=not symmetrize)


def sources(g: Graph, k: int, seed: int) -> np.ndarray:
    """k distinct seeded vertices of nonzero out-degree."""
    lib = _load()
    out = np.empty(max(k, 1), dtype=np.int32)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    got = lib.gg_sources(rp.ctypes.data, g.n, k, seed, out.ctypes.data)
    return out[:got].copy()


def rng_u64(seed: int, stream: int, i: int) -> int:
    return int(_load().gg_rng(seed, stream, i))


def ba_batch(g: int, nmin: int = 1000, nmax: int = 100000, m: int = 4, seed: int = 3) -> Batch:
    lib = _load()
    p = lib.gg_ba_batch(g, nmin, nmax, m, seed, _threads())
    if not p:
        raise MemoryError("ba_batch failed")
    try:
        G = lib.gg_batch_g(p)
        tn, te = lib.gg_batch_total_n(p), lib.gg_batch_total_nnz(p)
        vo = np.empty(G + 1, np.int64)
        eo = np.empty(G + 1, np.int64)
        rp = np.empty(tn + G, np.int64)
        col = np.empty(max(te, 1), np.int32)
        lib.gg_batch_copy(p, vo.ctypes.data, eo.ctypes.data, rp.ctypes.data, col.ctypes.data)
        return Batch(int(G), vo, eo, rp, col[:te])
    finally:
        lib.gg_batch_free(p)


# ---- small named graphs with closed-form BFS answers (test fixtures) ----

def path(n: int) -> Graph:
    u = np.arange(n - 1, dtype=np.int32)
    return from_edges(n, u, u + 1, True, f"path{n}")


def cycle(n: int) -> Graph:
    u = np.arange(n, dtype=np.int32)
    return from_edges(n, u, (u + 1) % n, True, f"cycle{n}")


def star(n: int) -> Graph:
    leaves = np.arange(1, n, dtype=np.int32)
    return from_edges(n, np.zeros(n - 1, np.int32), leaves, True, f"star{n}")


def complete(n: int) -> Graph:
    a, b = np.triu_indices(n, 1)
    return from_edges(n, a.astype(np.int32), b.astype(np.int32), True, f"complete{n}")


def lattice(rows: int, cols: int) -> Graph:
    """Unperturbed 4-neighbour lattice, vertex id r*cols + c."""
    return grid(rows, cols, 0.0, 0.0, seed=0)


def disjoint_union(*gs: Graph) -> Graph:
    us, vs, off = [], [], 0
    for g in gs:
        src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
        us.append((src + off).astype(np.int32))
        vs.append((g.col.astype(np.int64) + off).astype(np.int32))
        off += g.n
    g = from_edges(off, np.concatenate(us), np.concatenate(vs), False, "union")
    g.directed = any(x.directed for x in gs)
    return g
