"""Python binding of the GB300 BVSS BFS library (include/blest.h).

Argument marshalling only: every step of the BFS path runs in the CUDA
kernels of ``libblest.so``.  Arrays may be NumPy arrays (host) or torch
tensors (host or CUDA); outputs are written in place.  Importing this module
raises if the compiled library is missing -- build it first with
``python -c "import __graft_entry__ as g; g.build()"`` (or
``python paper_2606_05081_gb300/_build.py``).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import _build

LIB_PATH = _build.LIB

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libblest.so is not built ({LIB_PATH}); run paper_2606_05081_gb300/_build.py")

_lib = ctypes.CDLL(LIB_PATH)

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_INTERNAL = range(7)
REORDER_NONE, REORDER_RCM, REORDER_JACCARD, REORDER_AUTO = range(4)
MODE_PUSH_EAGER_CC, MODE_PUSH_EAGER_TC, MODE_PUSH_LAZY_CC, MODE_PUSH_LAZY_TC, MODE_BOTTOM_UP = range(5)
MODE_NAMES = ["push_eager_cc", "push_eager_tc", "push_lazy_cc", "push_lazy_tc", "bottom_up"]
POLICY_HEURISTIC, POLICY_LEARNED, POLICY_FIXED, POLICY_SCHEDULE = range(4)
NUM_CHOICES = 9   # learned-policy choices: modes 0-4 (lazy: 1 pass), 5/6 lazy CC 2/4 passes, 7/8 lazy TC 2/4
MLP_NW = 12 + 32 * 6 + 32 + 32 * 32 + 32 + NUM_CHOICES * 32 + NUM_CHOICES


def choice_mode_batch(c: int):
    """(mode, VSS passes in flight) of a learned-policy choice."""
    if c < 5:
        return c, 1
    return (2 if c < 7 else 3), (2 if (c - 5) % 2 == 0 else 4)


def choice_of(mode: int, batch: int) -> int:
    """The learned-policy choice of a mode run with `batch` passes in flight."""
    if mode in (MODE_PUSH_LAZY_CC, MODE_PUSH_LAZY_TC) and batch in (2, 4):
        return (5 if mode == MODE_PUSH_LAZY_CC else 7) + (0 if batch == 2 else 1)
    return mode


class BuildOpts(ctypes.Structure):
    _fields_ = [("reorder", ctypes.c_int32), ("sigma", ctypes.c_int32), ("directed", ctypes.c_int32),
                ("jaccard_window", ctypes.c_int32), ("probe_switch", ctypes.c_int32),
                ("engine_tc", ctypes.c_int32), ("eta", ctypes.c_float), ("udiv_threshold", ctypes.c_double),
                ("timeout_ms", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("vss_batch", ctypes.c_int32), ("tau", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("num_slice_sets", ctypes.c_int64),
                ("num_vss", ctypes.c_int64), ("num_slices", ctypes.c_int64),
                ("update_divergence", ctypes.c_double), ("lazy", ctypes.c_int32),
                ("switching", ctypes.c_int32), ("reorder", ctypes.c_int32), ("sigma", ctypes.c_int32),
                ("grid_blocks", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("build_ms", ctypes.c_double), ("device_bytes", ctypes.c_int64), ("tau", ctypes.c_int32),
                ("vss_batch", ctypes.c_int32), ("policy", ctypes.c_int32), ("engine_tc", ctypes.c_int32),
                ("model_loaded", ctypes.c_int32)]


class LevelLog(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int32), ("mode", ctypes.c_int32), ("frontier", ctypes.c_int64),
                ("frontier_edges", ctypes.c_int64), ("unvisited", ctypes.c_int64), ("queue", ctypes.c_int64),
                ("t_ns", ctypes.c_int64), ("scanned_vertices", ctypes.c_int64),
                ("scanned_arcs", ctypes.c_int64), ("slots", ctypes.c_int64), ("t_stage1_ns", ctypes.c_int64),
                ("vss_batch", ctypes.c_int64)]


class BvssView(ctypes.Structure):
    """blest_bvss_view: device pointers of a BVSS the caller owns."""
    _fields_ = [("n", ctypes.c_int64), ("num_slice_sets", ctypes.c_int64), ("num_vss", ctypes.c_int64),
                ("row_ids", ctypes.c_void_p), ("masks", ctypes.c_void_p), ("real_ptrs", ctypes.c_void_p),
                ("virtual_to_real", ctypes.c_void_p), ("out_degree", ctypes.c_void_p),
                ("engine_tc", ctypes.c_int32), ("sigma", ctypes.c_int32), ("tau", ctypes.c_int32)]


class DegreeReport(ctypes.Structure):
    """blest_degree_report: one degree distribution under the §4.2 footnote test."""
    _fields_ = [("top1", ctypes.c_double), ("top10", ctypes.c_double), ("gamma", ctypes.c_double),
                ("r2", ctypes.c_double), ("points", ctypes.c_int32), ("concentrated", ctypes.c_int32),
                ("powerlaw", ctypes.c_int32), ("heavy", ctypes.c_int32)]


class ScaleFreeReport(ctypes.Structure):
    """blest_scale_free_report."""
    _fields_ = [("out_deg", DegreeReport), ("in_deg", DegreeReport), ("scale_free", ctypes.c_int32)]


class MsbfsStats(ctypes.Structure):
    """blest_msbfs_stats: work counters of the last multi-source call."""
    _fields_ = [("kappa", ctypes.c_int64), ("launches", ctypes.c_int64), ("levels", ctypes.c_int64),
                ("vss", ctypes.c_int64), ("hit_words", ctypes.c_int64), ("dirty_sets", ctypes.c_int64),
                ("pull_levels", ctypes.c_int64), ("pull_arcs", ctypes.c_int64)]


_P = ctypes.c_void_p
_H = ctypes.c_void_p
_S = ctypes.c_int
_sigs = {
    "blest_default_opts": (None, [ctypes.POINTER(BuildOpts)]),
    "blest_build": (_S, [ctypes.c_int64, _P, _P, ctypes.POINTER(BuildOpts), ctypes.POINTER(_H)]),
    "blest_bfs": (_S, [_H, ctypes.c_int32, _P]),
    "blest_msbfs": (_S, [_H, _P, ctypes.c_int32, _P]),
    "blest_closeness": (_S, [_H, _P, _P, _P]),
    "blest_closeness_range": (_S, [_H, ctypes.c_int64, ctypes.c_int64, _P, _P]),
    "blest_build_many": (_S, [ctypes.c_int32, _P, _P, _P, _P, ctypes.POINTER(BuildOpts), ctypes.POINTER(_H)]),
    "blest_bfs_many": (_S, [_H, _P, _P]),
    "blest_set_policy": (_S, [_H, ctypes.c_int32, ctypes.c_int32]),
    "blest_set_schedule": (_S, [_H, _P, ctypes.c_int32]),
    "blest_set_engine": (_S, [_H, ctypes.c_int32]),
    "blest_set_launch": (_S, [_H, ctypes.c_int32, ctypes.c_int32]),
    "blest_set_switching": (_S, [_H, ctypes.c_int32]),
    "blest_set_queue_deferral": (_S, [_H, ctypes.c_int32]),
    "blest_set_msbfs_engine": (_S, [_H, ctypes.c_int32]),
    "blest_set_msbfs_variant": (_S, [_H, ctypes.c_int32, ctypes.c_int32]),
    "blest_set_msbfs_direction": (_S, [_H, ctypes.c_int32]),
    "blest_set_msbfs_output": (_S, [_H, ctypes.c_int32]),
    "blest_load_model": (_S, [_H, _P, ctypes.c_int32]),
    "blest_last_timings": (_S, [_H, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    "blest_get_info": (_S, [_H, ctypes.POINTER(Info)]),
    "blest_get_bvss": (_S, [_H, _P, _P, _P, _P]),
    "blest_get_perm": (_S, [_H, _P]),
    "blest_set_stream": (_S, [_H, _P, ctypes.c_int32]),
    "blest_sync": (_S, [_H]),
    "blest_destroy": (None, [_H]),
    "blest_status_string": (ctypes.c_char_p, [_S]),
    "blest_selftest_barrier_timeout": (_S, [ctypes.c_int32]),
    "blest_bfs_noalloc": (_S, [ctypes.POINTER(BvssView), ctypes.c_int32, _P, _P]),
    "blest_msbfs_stats": (_S, [_H, ctypes.POINTER(MsbfsStats)]),
    "blest_scale_free_test": (_S, [_P, _P, ctypes.c_int64, ctypes.POINTER(ScaleFreeReport)]),
    "blest_mlp_features": (_S, [_P, ctypes.c_int64, ctypes.c_float, _P]),
    "blest_mlp_loss_grad": (_S, [_P, _P, _P, ctypes.c_int64, _P, _P, _P]),
    "blest_mlp_train": (_S, [_P, _P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _P, _P]),
    "blest_mlp_predict": (_S, [_P, _P, ctypes.c_int64, _P, _P]),
    "blest_last_cuda_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = sorted(k for k in _sigs if k != "blest_last_cuda_error")


class BlestError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = _lib.blest_status_string(code).decode()
        extra = _lib.blest_last_cuda_error().decode() if code == ERR_CUDA else ""
        super().__init__(f"{what}: {msg} ({code}) {extra}".strip())
        self.code = code


def _check(code: int, what: str):
    if code != OK:
        raise BlestError(code, what)


def _ptr(a):
    """Raw pointer of a NumPy array or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _dtype_ok(a, np_dtype, torch_name):
    if hasattr(a, "data_ptr"):
        if str(a.dtype) != f"torch.{torch_name}":
            raise TypeError(f"expected torch.{torch_name}, got {a.dtype}")
    elif np.asarray(a).dtype != np_dtype:
        raise TypeError(f"expected {np_dtype}, got {np.asarray(a).dtype}")


def default_opts(**kw) -> BuildOpts:
    o = BuildOpts()
    _lib.blest_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Graph:
    """A built graph (one blest handle)."""

    def __init__(self, handle, n: int, many: bool = False):
        self._h = handle
        self.n = n
        self.many = many

    # ---------------------------------------------------------- lifetime
    def close(self):
        if self._h:
            _lib.blest_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -------------------------------------------------------------- BFS
    def bfs(self, source: int, out=None):
        """Levels from one source (int32, -1 = unreached); out may be a host
        array or a CUDA tensor of n int32."""
        if out is None:
            out = np.empty(self.n, np.int32)
        _dtype_ok(out, np.int32, "int32")
        _check(_lib.blest_bfs(self._h, int(source), _ptr(out)), "blest_bfs")
        return out

    def msbfs(self, sources, out=None):
        src = np.ascontiguousarray(sources, dtype=np.int32) if not hasattr(sources, "data_ptr") else sources
        k = len(src)
        if out is None:
            out = np.empty((k, self.n), np.int32)
        _dtype_ok(out, np.int32, "int32")
        _check(_lib.blest_msbfs(self._h, _ptr(src), k, _ptr(out)), "blest_msbfs")
        return out

    def closeness(self, far=None, cc=None, reach=None):
        if far is None:
            far = np.empty(self.n, np.int64)
        if cc is None:
            cc = np.empty(self.n, np.float64)
        if reach is None:
            reach = np.empty(self.n, np.int64)
        _check(_lib.blest_closeness(self._h, _ptr(far), _ptr(cc), _ptr(reach)), "blest_closeness")
        return far, cc, reach

    def closeness_range(self, first: int, count: int, far=None, reach=None):
        """Distance sums from the sources [first, first+count) only."""
        if far is None:
            far = np.empty(self.n, np.int64)
        if reach is None:
            reach = np.empty(self.n, np.int64)
        _check(_lib.blest_closeness_range(self._h, int(first), int(count), _ptr(far), _ptr(reach)),
               "blest_closeness_range")
        return far, reach

    def msbfs_stats(self) -> dict:
        """Work counters of the last multi-source or closeness call."""
        st = MsbfsStats()
        _check(_lib.blest_msbfs_stats(self._h, ctypes.byref(st)), "blest_msbfs_stats")
        return {f: int(getattr(st, f)) for f, _ in MsbfsStats._fields_}

    def bfs_many(self, sources, out=None, total_n=None):
        src = np.ascontiguousarray(sources, dtype=np.int32) if not hasattr(sources, "data_ptr") else sources
        if out is None:
            out = np.empty(int(total_n), np.int32)
        _check(_lib.blest_bfs_many(self._h, _ptr(src), _ptr(out)), "blest_bfs_many")
        return out

    # ---------------------------------------------------------- control
    def set_policy(self, policy: int, fixed_mode: int = 0):
        _check(_lib.blest_set_policy(self._h, policy, fixed_mode), "blest_set_policy")

    def set_engine(self, tc):
        """Top-down hit test: False / 0 CUDA cores, True / 1 the Fig. 3 b1-MMA
        layout, 2 the 16-MMA-per-VSS layout (ablation)."""
        _check(_lib.blest_set_engine(self._h, int(tc)), "blest_set_engine")

    def set_launch(self, block_threads: int, vss_batch: int):
        _check(_lib.blest_set_launch(self._h, int(block_threads), int(vss_batch)), "blest_set_launch")

    def set_msbfs_engine(self, tc: bool):
        """Multi-source stage 1 on the tensor cores (tcgen05, tau = 128) or
        on CUDA cores (the default)."""
        _check(_lib.blest_set_msbfs_engine(self._h, int(bool(tc))), "blest_set_msbfs_engine")

    def set_msbfs_direction(self, mode: int):
        """Multi-source stage 1: 0 push (Algorithm 5, the default), 1 pull on
        dense levels, 2 pull on every level."""
        _check(_lib.blest_set_msbfs_direction(self._h, int(mode)), "blest_set_msbfs_direction")

    def set_msbfs_output(self, staged: bool):
        """Multi-source levels staged as bytes in vertex-major rows and
        transposed at the end (the default), or one int32 store per reached
        (vertex, lane)."""
        _check(_lib.blest_set_msbfs_output(self._h, int(bool(staged))), "blest_set_msbfs_output")

    def set_msbfs_variant(self, reindex: bool = True, tracking: bool = True):
        """Multi-source kernel variant of the ablation: getVI reindexing and
        activeSets / dirtySets tracking on or off (both on = Algorithm 5)."""
        _check(_lib.blest_set_msbfs_variant(self._h, int(bool(reindex)), int(bool(tracking))),
               "blest_set_msbfs_variant")

    def set_switching(self, on: bool):
        """Eq. 5 bottom-up switching of the rule on or off (overrides the build's probe)."""
        _check(_lib.blest_set_switching(self._h, int(bool(on))), "blest_set_switching")

    def set_queue_deferral(self, mode: int):
        """Deferred VSS queues of lazy and bottom-up levels: 1 on, 0 off, -1
        (the default) on exactly when bottom-up switching is on."""
        _check(_lib.blest_set_queue_deferral(self._h, int(mode)), "blest_set_queue_deferral")

    def set_schedule(self, modes):
        m = np.ascontiguousarray(modes, dtype=np.int32)
        _check(_lib.blest_set_schedule(self._h, m.ctypes.data, len(m)), "blest_set_schedule")

    def load_model(self, weights):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        _check(_lib.blest_load_model(self._h, w.ctypes.data, len(w)), "blest_load_model")

    def set_stream(self, stream_ptr=None, async_: bool = False):
        _check(_lib.blest_set_stream(self._h, stream_ptr, int(async_)), "blest_set_stream")

    def sync(self):
        _check(_lib.blest_sync(self._h), "blest_sync")

    # ------------------------------------------------------ introspection
    def info(self) -> dict:
        i = Info()
        _check(_lib.blest_get_info(self._h, ctypes.byref(i)), "blest_get_info")
        return {f: getattr(i, f) for f, _ in Info._fields_}

    def level_log(self):
        n = ctypes.c_int64(0)
        _check(_lib.blest_last_timings(self._h, None, 0, ctypes.byref(n)), "blest_last_timings")
        buf = (LevelLog * max(1, n.value))()
        _check(_lib.blest_last_timings(self._h, buf, n.value, ctypes.byref(n)), "blest_last_timings")
        return [{f: getattr(buf[i], f) for f, _ in LevelLog._fields_} for i in range(n.value)]

    def bvss(self) -> dict:
        inf = self.info()
        nv, ns, tau = inf["num_vss"], inf["num_slice_sets"], inf["tau"]
        theta = 32 // inf["sigma"]
        rows = np.empty(nv * tau, np.int32)
        masks = np.empty(nv * tau // theta, np.uint32)
        real = np.empty(ns + 1, np.int32)
        v2r = np.empty(nv, np.int32)
        _check(_lib.blest_get_bvss(self._h, _ptr(rows), _ptr(masks), _ptr(real), _ptr(v2r)), "blest_get_bvss")
        return dict(rowIds=rows, masks=masks, realPtrs=real, v2r=v2r, Nv=nv, Ns=ns, sigma=inf["sigma"], tau=tau)

    def perm(self) -> np.ndarray:
        p = np.empty(self.n, np.int32)
        _check(_lib.blest_get_perm(self._h, _ptr(p)), "blest_get_perm")
        return p


def build(n: int, row_ptr, col_idx, **opts) -> Graph:
    """Build a handle from a CSR graph (host or device arrays).
    Options are the fields of blest_build_opts (reorder, directed, ...)."""
    _dtype_ok(row_ptr, np.int64, "int64")
    _dtype_ok(col_idx, np.int32, "int32")
    o = default_opts(**opts)
    h = _H()
    rp = row_ptr if hasattr(row_ptr, "data_ptr") else np.ascontiguousarray(row_ptr)
    ci = col_idx if hasattr(col_idx, "data_ptr") else np.ascontiguousarray(col_idx)
    if hasattr(ci, "data_ptr") and ci.numel() == 0 or (isinstance(ci, np.ndarray) and ci.size == 0):
        ci = np.zeros(1, np.int32)
    _check(_lib.blest_build(int(n), _ptr(rp), _ptr(ci), ctypes.byref(o), ctypes.byref(h)), "blest_build")
    return Graph(h, int(n))


def build_graph(g, **opts) -> Graph:
    """Build from a graphgen.Graph-like object (n, row_ptr, col, directed)."""
    if getattr(g, "directed", False):
        opts.setdefault("directed", 1)
    return build(g.n, g.row_ptr, g.col, **opts)


def build_many(batch, **opts) -> Graph:
    o = default_opts(**opts)
    h = _H()
    _check(_lib.blest_build_many(int(batch.g), _ptr(batch.vtx_off), _ptr(batch.edge_off), _ptr(batch.row_ptr),
                                 _ptr(batch.col), ctypes.byref(o), ctypes.byref(h)), "blest_build_many")
    return Graph(h, int(batch.vtx_off[-1]), many=True)


def selftest_barrier_timeout(timeout_ms: int = 20) -> int:
    return int(_lib.blest_selftest_barrier_timeout(int(timeout_ms)))


def scale_free_test(out_deg, in_deg=None) -> dict:
    """The §4.2 footnote's scale-free-like test on degree arrays (numpy or
    torch, host or device; in_deg None for an undirected graph)."""
    def arr(x):
        if x is None:
            return None
        if hasattr(x, "data_ptr"):
            import torch
            return x.to(dtype=torch.int32).contiguous()
        return np.ascontiguousarray(np.asarray(x), dtype=np.int32)
    o, i = arr(out_deg), arr(in_deg)
    rep = ScaleFreeReport()
    _check(_lib.blest_scale_free_test(_ptr(o), _ptr(i) if i is not None else None, len(o), ctypes.byref(rep)),
           "blest_scale_free_test")

    def d(r):
        return {f: getattr(r, f) for f, _ in DegreeReport._fields_}
    return {"out": d(rep.out_deg), "in": d(rep.in_deg), "scale_free": bool(rep.scale_free)}


def bfs_noalloc(view: BvssView, source: int, levels, stream=None):
    """Allocation-free BFS over a caller-held device BVSS (blest_bfs_noalloc).
    levels must be a CUDA int32 tensor of view.n elements."""
    _check(_lib.blest_bfs_noalloc(ctypes.byref(view), int(source), _ptr(levels), stream), "blest_bfs_noalloc")
    return levels


# ------------------------------------------------------------- learned policy
def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def mlp_features(records, avg_deg: float) -> np.ndarray:
    """Raw features (n, 6) of level-log records, computed by the device."""
    n = len(records)
    buf = (LevelLog * n)()
    for i, r in enumerate(records):
        for f, _ in LevelLog._fields_:
            setattr(buf[i], f, int(r[f]))
    out = np.empty((n, 6), np.float32)
    _check(_lib.blest_mlp_features(buf, n, float(avg_deg), out.ctypes.data), "blest_mlp_features")
    return out


def mlp_loss_grad(features, targets, mask, weights):
    _mlp_shapes(weights, features, targets, mask)
    X, T, M, W = _f32(features), _f32(targets), _f32(mask), _f32(weights)
    loss = ctypes.c_float(0)
    g = np.empty(MLP_NW, np.float32)
    _check(_lib.blest_mlp_loss_grad(X.ctypes.data, T.ctypes.data, M.ctypes.data, len(X), W.ctypes.data,
                                    ctypes.byref(loss), g.ctypes.data), "blest_mlp_loss_grad")
    return float(loss.value), g


def mlp_train(features, targets, mask, weights, epochs: int = 2000, lr: float = 1e-2, weight_decay: float = 0.0):
    _mlp_shapes(weights, features, targets, mask)
    X, T, M = _f32(features), _f32(targets), _f32(mask)
    W = _f32(weights).copy()
    hist = np.empty(epochs, np.float32)
    _check(_lib.blest_mlp_train(X.ctypes.data, T.ctypes.data, M.ctypes.data, len(X), int(epochs), float(lr),
                                float(weight_decay), W.ctypes.data, hist.ctypes.data), "blest_mlp_train")
    return W, hist


def _mlp_shapes(weights, features, targets=None, mask=None):
    """The C entry points cannot see buffer sizes: check them here."""
    if np.asarray(weights).size != MLP_NW:
        raise ValueError(f"weights: {MLP_NW} values expected")
    if np.asarray(features).ndim != 2 or np.asarray(features).shape[1] != 6:
        raise ValueError("features: shape (n, 6) expected")
    n = np.asarray(features).shape[0]
    for nm, a in (("targets", targets), ("mask", mask)):
        if a is not None and np.asarray(a).shape != (n, NUM_CHOICES):
            raise ValueError(f"{nm}: shape ({n}, {NUM_CHOICES}) expected")


def mlp_predict(weights, features):
    _mlp_shapes(weights, features)
    W, X = _f32(weights), _f32(features)
    pred = np.empty((len(X), NUM_CHOICES), np.float32)
    ch = np.empty(len(X), np.int32)
    _check(_lib.blest_mlp_predict(W.ctypes.data, X.ctypes.data, len(X), pred.ctypes.data, ch.ctypes.data),
           "blest_mlp_predict")
    return pred, ch
