"""CPU oracle for single-linkage dendrograms of weighted trees.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
GPU library never imports it and shares no code with it.

* ``dendrogram``: plain C Kruskal agglomeration (paper, Section 2.2.2, the
  bottom-up construction), ``kruskal.c``.
* ``dendrogram_batched``: the same, tree by tree, for offset-packed batches.
* ``edge_order``: the total order of edges (weight, -0.0 before +0.0, caller
  index), Section 3.1.
* ``cartesian_path``: closed form for path trees (Theorem 1), ``cartesian.c``.
* ``contraction``: a plain numpy model of the paper's alpha-edge contraction
  levels and multilevel expansion (Sections 3.2-3.3), for per-level checks.
* ``flat``: HDBSCAN* flat clusters of a dendrogram (the optional last step of
  the pipeline in Section 6.5, after Campello et al.), plain Python with exact
  rational sums.
* ``emst``: the mutual-reachability minimum spanning tree of a point set (the
  step before the dendrogram in Section 6.5), plain numpy, O(n^2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ("kruskal.c", "cartesian.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# status codes of the oracle (same meaning as the library's documented codes)
OK = 0
ERR_INVALID_ARGUMENT = 1
ERR_NAN_WEIGHT = 2
ERR_VERTEX_OUT_OF_RANGE = 3
ERR_SELF_LOOP = 4
ERR_NOT_A_TREE = 5
ERR_OUT_OF_MEMORY = 7


class OracleError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__(f"oracle status {code} {msg}".strip())
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle's C sources into ``liboracle.so`` (gcc, -O2)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        lib_m = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= lib_m for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", tmp] + srcs + \
        ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.oracle_dendrogram.argtypes = [p, p, p, i64, p, p]
            lib.oracle_dendrogram.restype = ctypes.c_int
            lib.oracle_dendrogram_batched.argtypes = [p, p, p, p, i64, p, p, p]
            lib.oracle_dendrogram_batched.restype = ctypes.c_int
            lib.oracle_edge_order.argtypes = [p, i64, p]
            lib.oracle_edge_order.restype = ctypes.c_int
            lib.oracle_dendrogram_threads.argtypes = [p, p, p, i64, p, p, ctypes.c_int]
            lib.oracle_dendrogram_threads.restype = ctypes.c_int
            lib.cartesian_path_dendrogram.argtypes = [p, p, i64, p, p]
            lib.cartesian_path_dendrogram.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _as(a, dtype):
    return np.ascontiguousarray(np.asarray(a), dtype=dtype)


def dendrogram(u, v, w, check: bool = True):
    """(edge_parent, vertex_parent) of one tree, or raises ``OracleError``.

    With ``check=False`` returns ``(status, edge_parent, vertex_parent)``.
    """
    lib = _load()
    u = _as(u, np.int32)
    v = _as(v, np.int32)
    w = _as(w, np.float32)
    m = int(w.shape[0])
    ep = np.empty(max(m, 1), np.int32)
    vp = np.empty(m + 1, np.int32)
    st = lib.oracle_dendrogram(_ptr(u), _ptr(v), _ptr(w), m, _ptr(ep), _ptr(vp))
    ep = ep[:m]
    if not check:
        return st, ep, vp
    if st != OK:
        raise OracleError(st)
    return ep, vp


def dendrogram_threads(u, v, w, n_threads: int):
    """The same dendrogram with the edge sort on ``n_threads`` threads and the
    union-find pass sequential (the all-core timing mode); raises
    ``OracleError``."""
    lib = _load()
    u = _as(u, np.int32)
    v = _as(v, np.int32)
    w = _as(w, np.float32)
    m = int(w.shape[0])
    ep = np.empty(max(m, 1), np.int32)
    vp = np.empty(m + 1, np.int32)
    st = lib.oracle_dendrogram_threads(_ptr(u), _ptr(v), _ptr(w), m, _ptr(ep), _ptr(vp),
                                       int(n_threads))
    if st != OK:
        raise OracleError(st)
    return ep[:m], vp


def dendrogram_batched(u, v, w, edge_offsets, check: bool = True):
    """Tree-local (edge_parent, vertex_parent) for an offset-packed batch."""
    lib = _load()
    u = _as(u, np.int32)
    v = _as(v, np.int32)
    w = _as(w, np.float32)
    off = _as(edge_offsets, np.int64)
    t = int(off.shape[0]) - 1
    m = int(off[-1])
    ep = np.empty(max(m, 1), np.int32)
    vp = np.empty(m + t, np.int32)
    bad = np.full(1, -1, np.int64)
    st = lib.oracle_dendrogram_batched(_ptr(u), _ptr(v), _ptr(w), _ptr(off), t, _ptr(ep),
                                       _ptr(vp), _ptr(bad))
    ep = ep[:m]
    if not check:
        return st, ep, vp
    if st != OK:
        raise OracleError(st, f"(tree {int(bad[0])})")
    return ep, vp


def edge_order(w) -> np.ndarray:
    """Caller indices of the edges from lightest to heaviest."""
    lib = _load()
    w = _as(w, np.float32)
    order = np.empty(max(int(w.shape[0]), 1), np.int32)
    st = lib.oracle_edge_order(_ptr(w), int(w.shape[0]), _ptr(order))
    if st != OK:
        raise OracleError(st)
    return order[: w.shape[0]]


def cartesian_path(w_path, eid):
    """Closed-form dendrogram of a path (Theorem 1).

    ``w_path[k]`` and ``eid[k]`` are the weight and caller index of the k-th
    edge along the path.  Returns ``(edge_parent, vertex_parent_path)`` where
    ``vertex_parent_path[k]`` is the parent of the k-th path vertex.
    """
    lib = _load()
    wp = _as(w_path, np.float32)
    eid = _as(eid, np.int32)
    m = int(wp.shape[0])
    ep = np.empty(max(m, 1), np.int32)
    vpp = np.empty(m + 1, np.int32)
    st = lib.cartesian_path_dendrogram(_ptr(wp), _ptr(eid), m, _ptr(ep), _ptr(vpp))
    if st != 0:
        raise OracleError(st)
    return ep[:m], vpp
