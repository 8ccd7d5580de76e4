"""ctypes binding of libsimrank (include/simrank.h): argument marshalling only.

Every computation happens inside the CUDA library; this module converts
NumPy / torch arguments to plain pointers and status codes to exceptions.
It raises if the in-tree library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsimrank.so")

SR_OK = 0
STATUS_NAMES = {
    0: "SR_OK", 1: "SR_ERR_ARG", 2: "SR_ERR_EDGE_EXISTS", 3: "SR_ERR_EDGE_MISSING",
    4: "SR_ERR_CAPACITY", 5: "SR_ERR_OOM", 6: "SR_ERR_CUDA", 7: "SR_ERR_TIMEOUT",
    8: "SR_ERR_NOT_CONVERGED", 9: "SR_ERR_UNSUPPORTED",
}
MODE_DENSE, MODE_COLUMN = 0, 1
APPLY_UNIT, APPLY_SINK_BLOCKS, APPLY_ONE_SHOT = 0, 1, 2
SUPDATE_FUSED, SUPDATE_PLAIN = 0, 1
INIT_SWEEPS, INIT_FOREST, INIT_COMPONENTS = 0, 1, 2


class SimrankError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [
        ("C", ctypes.c_double), ("K", ctypes.c_int32), ("s_precision", ctypes.c_int32),
        ("mode", ctypes.c_int32), ("n_capacity", ctypes.c_int32), ("aff", ctypes.c_int32),
        ("apply", ctypes.c_int32), ("s_update", ctypes.c_int32), ("tc", ctypes.c_int32),
        ("init_max_sweeps", ctypes.c_int32), ("init_tol", ctypes.c_double),
        ("profile", ctypes.c_int32), ("relabel", ctypes.c_int32),
        ("timeout_iters", ctypes.c_int64), ("cuda_stream", ctypes.c_void_p),
        ("s_kernel", ctypes.c_int32), ("defer", ctypes.c_int32), ("chain", ctypes.c_int32),
        ("prep_ctas", ctypes.c_int32), ("prep_cache", ctypes.c_int32),
        ("multi_launch", ctypes.c_int32), ("prep_item", ctypes.c_int32),
        ("upper_only", ctypes.c_int32), ("vec_fp64", ctypes.c_int32),
        ("init_form", ctypes.c_int32), ("reanchor_every", ctypes.c_int32),
        ("reanchor_sweeps", ctypes.c_int32),
    ]


class Update(ctypes.Structure):
    _fields_ = [("src", ctypes.c_int32), ("dst", ctypes.c_int32), ("op", ctypes.c_int32),
                ("weight", ctypes.c_float)]


class Stats(ctypes.Structure):
    _fields_ = [
        ("updates", ctypes.c_int64), ("rank_one_updates", ctypes.c_int64),
        ("tiles_total", ctypes.c_int64), ("tiles_touched", ctypes.c_int64),
        ("s_bytes", ctypes.c_int64), ("panel_bytes", ctypes.c_int64),
        ("s_update_launches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
        ("s_update_ms", ctypes.c_double),
        ("init_residual", ctypes.c_double), ("phase_ms", ctypes.c_double * 4),
        ("init_sweeps", ctypes.c_int32), ("reanchors", ctypes.c_int32),
        ("reanchor_residual", ctypes.c_double), ("reanchor_change", ctypes.c_double),
        ("reserved", ctypes.c_int32 * 2),
    ]


UPDATE_DTYPE = np.dtype([("src", np.int32), ("dst", np.int32), ("op", np.int32), ("weight", np.float32)])

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

# name -> (restype, argtypes); every symbol declared in include/simrank.h
SIGNATURES = {
    "simrank_default_config": (_I32, [ctypes.POINTER(Config)]),
    "simrank_init": (_I32, [ctypes.POINTER(Config), _I32, _I64, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "simrank_apply_updates": (_I32, [_P, _P, _I64]),
    "simrank_columns": (_I32, [_P, _P, _I32, _P, _I32, _I32]),
    "simrank_num_nodes": (_I32, [_P]),
    "simrank_last_error": (ctypes.c_char_p, [_P]),
    "simrank_sync": (_I32, [_P]),
    "simrank_destroy": (None, [_P]),
    "simrank_get_stats": (_I32, [_P, ctypes.POINTER(Stats)]),
    "simrank_reanchor": (_I32, [_P, _I32, ctypes.POINTER(ctypes.c_double)]),
    "simrank_set_launch": (_I32, [_P, ctypes.POINTER(Config)]),
    "simrank_plan_batch": (_I32, [_P, _I64, _I32, _I32, ctypes.POINTER(_I32), _P, _P, _P, _P]),
    "simrank_grad": (_I32, [_P, _P, _P, _P, _I64, ctypes.POINTER(ctypes.c_double), _P]),
    "simrank_update_noalloc": (_I32, [_I32, _I64, _P, _I32, _P, _P, _P, _P, _I32, _I32, _I32, _I32,
                                      ctypes.c_double, _I32, _P]),
    "simrank_multi_init": (_I32, [ctypes.POINTER(Config), _I32, _P, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "simrank_multi_apply": (_I32, [_P, _P, _P]),
    "simrank_multi_columns": (_I32, [_P, _I32, _P, _I32, _P, _I32, _I32]),
    "simrank_multi_num_graphs": (_I32, [_P]),
    "simrank_multi_num_nodes": (_I32, [_P, _I32]),
    "simrank_multi_sync": (_I32, [_P]),
    "simrank_multi_get_stats": (_I32, [_P, ctypes.POINTER(Stats)]),
    "simrank_multi_last_error": (ctypes.c_char_p, [_P]),
    "simrank_multi_destroy": (None, [_P]),
}

_lib = None


def lib():
    """Loads the in-tree libsimrank.so (build it with __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libsimrank.so not built at {LIB_PATH}; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(status, handle=None):
    if status != SR_OK:
        msg = lib().simrank_last_error(handle)
        raise SimrankError(status, msg.decode() if msg else "")


def default_config(**kw) -> Config:
    cfg = Config()
    _check(lib().simrank_default_config(ctypes.byref(cfg)))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise TypeError(f"unknown config field {k}")
        setattr(cfg, k, v)
    return cfg


def updates_array(upd) -> np.ndarray:
    """(count, 3) int array of (src, dst, op) -> packed simrank_update records."""
    upd = np.asarray(upd)
    out = np.zeros(upd.shape[0], UPDATE_DTYPE)
    if upd.shape[0]:
        out["src"] = upd[:, 0]
        out["dst"] = upd[:, 1]
        out["op"] = upd[:, 2]
    return out


class SimRank:
    """Handle on a graph and its SimRank matrix in GPU memory."""

    def __init__(self, n, src, dst, weight=None, S0=None, stream=None, tuned=False, **cfg_kw):
        """cfg_kw: simrank_config fields.  tuned=True takes the launch knobs the
        autotuner cached for this GPU and shape (paper_1711_00121_gb300.tune)
        for every knob not given explicitly."""
        self._h = None
        if tuned:
            from .tune import tuned_knobs

            probe = default_config(**cfg_kw)
            for k, v in tuned_knobs("stream", n, probe.K, probe.s_precision, probe.vec_fp64).items():
                cfg_kw.setdefault(k, v)
        self.tuned_config = dict(cfg_kw)
        cfg = default_config(**cfg_kw)
        if stream is not None:
            cfg.cuda_stream = stream
        src = np.ascontiguousarray(src, np.int32)
        dst = np.ascontiguousarray(dst, np.int32)
        w = None if weight is None else np.ascontiguousarray(weight, np.float32)
        s0 = None
        if S0 is not None:
            s0 = np.ascontiguousarray(S0, np.float64 if cfg.s_precision == 64 else np.float32)
        h = ctypes.c_void_p()
        st = lib().simrank_init(ctypes.byref(cfg), int(n), int(src.size), _ptr(src), _ptr(dst),
                                _ptr(w), _ptr(s0), ctypes.byref(h))
        _check(st, None)
        self._h = h
        self.config = cfg

    def close(self):
        if self._h is not None:
            lib().simrank_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return int(lib().simrank_num_nodes(self._h))

    def apply_updates(self, upd):
        """Apply (src, dst, op) rows, or a packed simrank_update array."""
        arr = upd if (isinstance(upd, np.ndarray) and upd.dtype == UPDATE_DTYPE) else updates_array(upd)
        arr = np.ascontiguousarray(arr)
        _check(lib().simrank_apply_updates(self._h, _ptr(arr), int(arr.size)), self._h)

    def apply_updates_ptr(self, ptr, count):
        """Apply `count` packed updates at a host address (e.g. pinned memory)."""
        _check(lib().simrank_apply_updates(self._h, ctypes.c_void_p(ptr), int(count)), self._h)

    def columns(self, cols, fp64=True):
        """Columns of S as a host array of shape (n, len(cols))."""
        cols = np.ascontiguousarray(cols, np.int32)
        n = self.n
        out = np.empty((cols.size, n), np.float64 if fp64 else np.float32)
        _check(lib().simrank_columns(self._h, _ptr(cols), int(cols.size), _ptr(out), 0, int(fp64)), self._h)
        return out.T

    def columns_device(self, cols, out):
        """Columns into a device tensor `out` (torch, shape (len(cols), n), float32/64)."""
        cols = np.ascontiguousarray(cols, np.int32)
        fp64 = 1 if str(out.dtype).endswith("float64") else 0
        _check(lib().simrank_columns(self._h, _ptr(cols), int(cols.size), _ptr(out), 1, fp64), self._h)

    def dense(self, fp64=True):
        """The whole current S (n x n) on the host."""
        return self.columns(np.arange(self.n, dtype=np.int32), fp64=fp64)

    def sync(self):
        _check(lib().simrank_sync(self._h), self._h)

    def stats(self) -> dict:
        s = Stats()
        _check(lib().simrank_get_stats(self._h, ctypes.byref(s)), self._h)
        out = {name: getattr(s, name) for name, _ in Stats._fields_ if name != "reserved"}
        out["phase_ms"] = list(s.phase_ms)
        return out

    def grad(self, a, b, target, m):
        """Pair loss and its gradient with respect to the m initial edge weights."""
        a = np.ascontiguousarray(a, np.int32)
        b = np.ascontiguousarray(b, np.int32)
        t = np.ascontiguousarray(target, np.float64)
        g = np.zeros(int(m), np.float64)
        L = ctypes.c_double()
        _check(lib().simrank_grad(self._h, _ptr(a), _ptr(b), _ptr(t), int(a.size), ctypes.byref(L),
                                  _ptr(g)), self._h)
        return L.value, g

    def set_launch(self, **knobs):
        """Changes the launch shape of later updates (defer, tc, prep_ctas,
        prep_cache, prep_item, s_kernel); other config fields keep their values."""
        cfg = Config()
        ctypes.memmove(ctypes.byref(cfg), ctypes.byref(self.config), ctypes.sizeof(Config))
        for k, v in knobs.items():
            setattr(cfg, k, v)
        _check(lib().simrank_set_launch(self._h, ctypes.byref(cfg)), self._h)
        for k, v in knobs.items():
            setattr(self.config, k, v)

    def reanchor(self, sweeps):
        d = ctypes.c_double()
        _check(lib().simrank_reanchor(self._h, int(sweeps), ctypes.byref(d)), self._h)
        return d.value


def _mcheck(status, handle=None):
    if status != SR_OK:
        msg = lib().simrank_multi_last_error(handle)
        raise SimrankError(status, msg.decode() if msg else "")


class MultiSimRank:
    """Many independent graphs in GPU memory, advanced together.

    ``graphs`` is a list of (n, src, dst) or (n, src, dst, n_capacity).
    """

    def __init__(self, graphs, stream=None, tuned=False, **cfg_kw):
        """graphs as above; cfg_kw: simrank_config fields; tuned=True takes the
        S-pass form the autotuner cached for this GPU (unless tc is given)."""
        if tuned:
            from .tune import tuned_knobs

            probe = default_config(**cfg_kw)
            nmax = max(int(gr[0]) for gr in graphs)
            for k, v in tuned_knobs("multi", nmax, probe.K, probe.s_precision, 0).items():
                cfg_kw.setdefault(k, v)
        self.tuned_config = dict(cfg_kw)
        cfg = default_config(**cfg_kw)
        if stream is not None:
            cfg.cuda_stream = stream
        n = np.array([int(gr[0]) for gr in graphs], np.int32)
        cap = np.array([int(gr[3]) if len(gr) > 3 else int(gr[0]) for gr in graphs], np.int32)
        m = [len(gr[1]) for gr in graphs]
        off = np.zeros(len(graphs) + 1, np.int64)
        off[1:] = np.cumsum(m)
        src = np.ascontiguousarray(np.concatenate([np.asarray(gr[1], np.int32) for gr in graphs]))
        dst = np.ascontiguousarray(np.concatenate([np.asarray(gr[2], np.int32) for gr in graphs]))
        h = _P()
        _mcheck(lib().simrank_multi_init(ctypes.byref(cfg), len(graphs), _ptr(n), _ptr(cap), _ptr(off),
                                         _ptr(src), _ptr(dst), ctypes.byref(h)), None)
        self._h = h
        self.cfg = cfg

    @property
    def num_graphs(self):
        return lib().simrank_multi_num_graphs(self._h)

    def num_nodes(self, g):
        return lib().simrank_multi_num_nodes(self._h, int(g))

    def apply_updates(self, per_graph):
        """per_graph[g]: (count, 3) array of (src, dst, op) for graph g."""
        arrs = [updates_array(np.asarray(x).reshape(-1, 3)) for x in per_graph]
        off = np.zeros(len(arrs) + 1, np.int64)
        off[1:] = np.cumsum([a.size for a in arrs])
        allu = np.ascontiguousarray(np.concatenate(arrs)) if arrs else np.zeros(0, UPDATE_DTYPE)
        self.apply_packed(allu, off)

    def apply_packed(self, packed, offsets):
        """Packed simrank_update records (host) and their ngraphs + 1 offsets."""
        _mcheck(lib().simrank_multi_apply(self._h, _ptr(packed), _ptr(offsets)), self._h)

    def columns(self, g, cols, fp64=True):
        cols = np.ascontiguousarray(cols, np.int32)
        n = self.num_nodes(g)
        out = np.zeros((cols.size, n), np.float64 if fp64 else np.float32)
        _mcheck(lib().simrank_multi_columns(self._h, int(g), _ptr(cols), int(cols.size), _ptr(out), 0,
                                            1 if fp64 else 0), self._h)
        return out.T

    def dense(self, g, fp64=True):
        return self.columns(g, np.arange(self.num_nodes(g), dtype=np.int32), fp64=fp64)

    def sync(self):
        _mcheck(lib().simrank_multi_sync(self._h), self._h)

    def stats(self) -> dict:
        s = Stats()
        _mcheck(lib().simrank_multi_get_stats(self._h, ctypes.byref(s)), self._h)
        out = {name: getattr(s, name) for name, _ in Stats._fields_ if name != "reserved"}
        out["phase_ms"] = list(s.phase_ms)
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().simrank_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_batch(upd, n_old):
    """Host-only §8 batch planning; returns a list of (sink, op, [sources])."""
    arr = np.ascontiguousarray(updates_array(upd))
    cnt = arr.size
    nb = ctypes.c_int32()
    sink = np.zeros(max(cnt, 1), np.int32)
    op = np.zeros(max(cnt, 1), np.int32)
    off = np.zeros(max(cnt, 1) + 1, np.int64)
    srcs = np.zeros(max(cnt, 1), np.int32)
    st = lib().simrank_plan_batch(_ptr(arr), int(cnt), int(n_old), int(max(cnt, 1)), ctypes.byref(nb),
                                  _ptr(sink), _ptr(op), _ptr(off), _ptr(srcs))
    _check(st, None)
    return [(int(sink[b]), int(op[b]), srcs[off[b]:off[b + 1]].tolist()) for b in range(nb.value)]
