"""CPU oracle for the BVSS BFS path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library (``include/blest.h`` and
``paper_2606_05081_gb300``) never imports, links or calls it, and it shares
no code with the GPU path; the two meet only through the seeded inputs of
``graphgen``.

Contents (each function cites the passage of the paper it restates):
  bfs / bfs_many        serial FIFO queue BFS levels (C, ``bfs_oracle.c``), §2 Eq. 1
  far_reach / closeness per-vertex distance sums and closeness, §6.2 Eq. 6-7
  bvss                  the BVSS arrays of §3.1 written out from the definition
  update_divergence     U_div of §4.2
  get_vi                the MS-BFS vertex remap of §6.1
  mma_m8n8k128_b1       the binary MMA (popc, and) of §2.1 on lane registers
  paper_frag_b          the fragB register layout of Fig. 3
  gteps_edges           the edge count used for TEPS (a reading; the paper
                        defines none)
  classify (module)     the scale-free-like test of the §4.2 footnote
  reorder (module)      RCM (§4.2) and JaccardWithWindows (Algorithm 1)
  mlp (module)          the level-mode MLP, its loss, gradient and Adam
Every function here is pinned by tests in ``tests/test_oracle_*.py`` against
closed forms, library routines, brute force or values printed in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P, i64, i32, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int
            lib.or_bfs.restype = ci
            lib.or_bfs.argtypes = [i64, P, P, i32, P]
            lib.or_bfs_many.restype = ci
            lib.or_bfs_many.argtypes = [i64, P, P, i32, P, P, ci]
            lib.or_far_reach.restype = ci
            lib.or_far_reach.argtypes = [i64, P, P, i32, P, P, P, ci]
            _lib = lib
    return _lib


def _threads(nthreads):
    return nthreads if nthreads else max(1, os.cpu_count() or 1)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, np.int32)
    return rp, col


# --------------------------------------------------------------- BFS levels
def bfs(g, src: int) -> np.ndarray:
    """Levels from one source (§2, Eq. 1): hop distance, -1 if unreachable."""
    rp, col = _csr(g)
    out = np.empty(g.n, np.int32)
    if _load().or_bfs(g.n, rp.ctypes.data, col.ctypes.data, int(src), out.ctypes.data):
        raise ValueError("invalid source")
    return out


def bfs_many(g, srcs, nthreads: int = 0) -> np.ndarray:
    """One serial BFS per source; returns levels[k, n] (source-major)."""
    rp, col = _csr(g)
    s = np.ascontiguousarray(srcs, dtype=np.int32)
    out = np.empty((len(s), g.n), np.int32)
    if len(s) and _load().or_bfs_many(g.n, rp.ctypes.data, col.ctypes.data, len(s), s.ctypes.data,
                                     out.ctypes.data, _threads(nthreads)):
        raise ValueError("invalid source")
    return out


# --------------------------------------------------------------- closeness
def far_reach(g, verts=None, nthreads: int = 0):
    """far[i] = sum of hop distances from verts[i] to every vertex it reaches,
    reach[i] = number of vertices it reaches (itself included).  On an
    undirected graph this equals the per-target sum of Eq. 6 (§6.2)."""
    rp, col = _csr(g)
    if verts is None:
        verts = np.arange(g.n, dtype=np.int32)
    v = np.ascontiguousarray(verts, dtype=np.int32)
    far = np.zeros(len(v), np.int64)
    reach = np.zeros(len(v), np.int64)
    if len(v) and _load().or_far_reach(g.n, rp.ctypes.data, col.ctypes.data, len(v), v.ctypes.data,
                                      far.ctypes.data, reach.ctypes.data, _threads(nthreads)):
        raise ValueError("invalid vertex")
    return far, reach


def closeness_from(far: np.ndarray, reach: np.ndarray) -> np.ndarray:
    """Eq. 7 with the component-size normalisation §6.2 allows for a
    disconnected graph: cc = (reach - 1) / far, 0 where far == 0.  On a
    connected graph reach = n, which is Eq. 7 exactly."""
    far = np.asarray(far, np.int64)
    cc = np.zeros(far.shape, np.float64)
    nz = far > 0
    cc[nz] = (np.asarray(reach, np.int64)[nz] - 1).astype(np.float64) / far[nz].astype(np.float64)
    return cc


def closeness(g, nthreads: int = 0):
    far, reach = far_reach(g, None, nthreads)
    return far, reach, closeness_from(far, reach)


# --------------------------------------------------------------- BVSS (§3.1)
def bvss(g, sigma: int = 8, tau: int | None = None) -> dict:
    """The BVSS arrays of §3.1, built from their definition.

    A is the transposed adjacency (§2): A[i][j] = 1 iff (j, i) is an arc, so
    the nonzeros of column j are the out-neighbours of j (CSR row j).  Slice
    set s covers columns [s*sigma, (s+1)*sigma); its slices are the rows with
    a nonzero there, each with a sigma-bit mask (bit j - s*sigma, least
    significant bit first, the convention of Fig. 1).  Slices of a slice set
    are kept in ascending row order (a choice; the paper leaves the order
    open).  A 32-bit word holds theta = 32/sigma masks.  Each slice set is
    cut into VSSs of at most tau slices -- by default tau = 32*theta, one
    word per lane of a warp; tau = 32 with sigma = 8 gives VSSs of eight
    lane words -- and the last VSS of a set is padded with zero masks and
    row id 0.  Slice k of VSS v sits at slot v*tau + k, so lane word l of
    the VSS owns slots v*tau + l*theta + c, c < theta, and holds mask c in
    bits [c*sigma, (c+1)*sigma).  realPtrs (N_s + 1) maps a slice set to its
    VSS range; virtualToReal (N_v) maps back.  Slice sets with no slice get
    no VSS.
    """
    assert sigma in (8, 16, 32)
    theta = 32 // sigma
    if tau is None:
        tau = 32 * theta
    assert tau % theta == 0 and tau in (32, 64, 128)
    lanes = tau // theta
    n = g.n
    Ns = (n + sigma - 1) // sigma
    deg = np.diff(g.row_ptr).astype(np.int64)
    j = np.repeat(np.arange(n, dtype=np.int64), deg)       # column of each nonzero
    i = np.asarray(g.col, dtype=np.int64)                   # row of each nonzero
    s = j // sigma
    key = s * n + i
    uk, inv = np.unique(key, return_inverse=True)           # sorted by (slice set, row)
    smask = np.zeros(len(uk), np.uint64)
    np.bitwise_or.at(smask, inv, (np.uint64(1) << (j % sigma).astype(np.uint64)))
    slice_set = uk // n
    slice_row = uk % n
    count = np.bincount(slice_set, minlength=Ns).astype(np.int64)
    nvss = (count + tau - 1) // tau
    realPtrs = np.zeros(Ns + 1, np.int64)
    realPtrs[1:] = np.cumsum(nvss)
    Nv = int(realPtrs[-1])
    v2r = np.repeat(np.arange(Ns, dtype=np.int64), nvss)
    first = np.zeros(Ns + 1, np.int64)
    first[1:] = np.cumsum(count)
    rank = np.arange(len(uk), dtype=np.int64) - first[slice_set]
    slot = (realPtrs[slice_set] + rank // tau) * tau + rank % tau
    rowIds = np.zeros(Nv * tau, np.int64)
    rowIds[slot] = slice_row
    mslot = np.zeros(Nv * tau, np.uint64)
    mslot[slot] = smask
    shifts = (np.arange(theta, dtype=np.uint64) * np.uint64(sigma))
    masks = np.bitwise_or.reduce(mslot.reshape(Nv * lanes, theta) << shifts, axis=1) if Nv else \
        np.zeros(0, np.uint64)
    return dict(sigma=sigma, theta=theta, tau=tau, lanes=lanes, n=n, Ns=Ns, Nv=Nv,
                rowIds=rowIds.astype(np.int32), masks=masks.astype(np.uint32),
                slot_masks=mslot.astype(np.uint32),
                realPtrs=realPtrs.astype(np.int32), v2r=v2r.astype(np.int32),
                num_slices=int(len(uk)))


def update_divergence(b: dict) -> float:
    """U_div of §4.2: for each VSS, each of its theta columns (the slices a
    lane word holds at position c, over the VSS's lane words) has a column
    divergence = population standard deviation of the row ids whose masks
    are nonzero; the set divergence averages it over the non-empty columns;
    U_div averages the set divergence over all N_v VSSs."""
    Nv, theta, lanes = b["Nv"], b["theta"], b["lanes"]
    if Nv == 0:
        return 0.0
    R = b["rowIds"].astype(np.float64).reshape(Nv, lanes, theta)
    M = (b["slot_masks"].reshape(Nv, lanes, theta) != 0)
    cnt = M.sum(axis=1)                                        # [Nv, theta]
    safe = np.maximum(cnt, 1)
    mean = (R * M).sum(axis=1) / safe
    var = (((R - mean[:, None, :]) ** 2) * M).sum(axis=1) / safe
    std = np.sqrt(var)
    nonempty = cnt > 0
    setdiv = (std * nonempty).sum(axis=1) / np.maximum(nonempty.sum(axis=1), 1)
    return float(setdiv.mean())


# ------------------------------------------------------------ getVI (§6.1)
def get_vi(u, rho: int, sigma: int = 8):
    """getVI(u, rho) = (u mod sigma) * rho + floor(u / sigma) (§6.1)."""
    u = np.asarray(u, dtype=np.int64)
    return (u % sigma) * rho + u // sigma


# ------------------------------------------------- binary MMA (§2.1, Fig. 3)
def _popc32(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    return np.array([bin(int(v)).count("1") for v in x.ravel()], dtype=np.int64).reshape(x.shape)


def mma_m8n8k128_b1(a_regs, b_regs, c_regs=None) -> np.ndarray:
    """D = A (.) B + C over the (popc, and) semiring of §2.1 for the
    m8n8k128 binary shape.  Register ownership follows the PTX ISA fragment
    layout of that shape: lane t holds A row t//4, bits 32*(t%4)..+31; B
    column t//4, bits 32*(t%4)..+31; D row t//4, columns 2*(t%4) and
    2*(t%4)+1.  Returns d_regs[32, 2]."""
    a = np.asarray(a_regs, dtype=np.uint64).reshape(32)
    b = np.asarray(b_regs, dtype=np.uint64).reshape(32)
    A = np.zeros((8, 4), np.uint64)
    Bc = np.zeros((8, 4), np.uint64)          # Bc[col][word]
    for t in range(32):
        A[t // 4, t % 4] = a[t]
        Bc[t // 4, t % 4] = b[t]
    D = np.zeros((8, 8), np.int64)
    for i in range(8):
        for jj in range(8):
            D[i, jj] = int(_popc32(A[i] & Bc[jj]).sum())
    out = np.zeros((32, 2), np.int64)
    for t in range(32):
        out[t, 0] = D[t // 4, 2 * (t % 4)]
        out[t, 1] = D[t // 4, 2 * (t % 4) + 1]
    if c_regs is not None:
        out += np.asarray(c_regs, dtype=np.int64).reshape(32, 2)
    return out


def paper_frag_b(alpha: int) -> np.ndarray:
    """fragB registers of Fig. 3 for a sigma=8 frontier byte alpha: lanes
    with t mod 9 == 0 hold X Z = alpha, lanes with t mod 9 == 4 hold
    Y Z = alpha << 8, all others zero (§5.1)."""
    b = np.zeros(32, np.uint64)
    for t in range(32):
        if t % 9 == 0:
            b[t] = alpha & 0xFF
        elif t % 9 == 4:
            b[t] = (alpha & 0xFF) << 8
    return b


def slice_hits(mask_words, alpha: int, sigma: int = 8) -> np.ndarray:
    """Eq. 2 per slice: hit = popc(mask & alpha) > 0 for each of the theta
    masks in each lane word.  Returns bool[len(mask_words), theta]."""
    theta = 32 // sigma
    w = np.asarray(mask_words, dtype=np.uint64)
    full = np.uint64((1 << sigma) - 1)
    out = np.zeros((len(w), theta), bool)
    for c in range(theta):
        m = (w >> np.uint64(c * sigma)) & full
        out[:, c] = _popc32(m & np.uint64(alpha)) > 0
    return out


# ----------------------------------------------------------------- TEPS
def gteps_edges(g, levels: np.ndarray) -> int:
    """Edges traversed by one BFS, for TEPS (a reading: the paper defines no
    TEPS).  Graph500 convention: arcs leaving reached vertices, halved on an
    undirected graph so each edge counts once."""
    deg = np.diff(g.row_ptr)
    arcs = int(deg[np.asarray(levels) >= 0].sum())
    return arcs if g.directed else arcs // 2
