"""ctypes binding of libpandora.so (argument marshalling only).

Every function here checks its tensors, hands raw device pointers and the
current CUDA stream to the C ABI of ``include/pandora.h`` and raises
``PandoraError`` on a non-zero status.  No step of the dendrogram is computed
in Python, and there is no CPU fallback: without the library or a GPU the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_NAME = "libpandora.so"
_lock = threading.Lock()
_lib = None

MAX_LEVELS = 64

STATUS_NAMES = {
    0: "PANDORA_OK",
    1: "PANDORA_ERR_INVALID_ARGUMENT",
    2: "PANDORA_ERR_NAN_WEIGHT",
    3: "PANDORA_ERR_VERTEX_OUT_OF_RANGE",
    4: "PANDORA_ERR_SELF_LOOP",
    5: "PANDORA_ERR_NOT_A_TREE",
    6: "PANDORA_ERR_ITERATION_LIMIT",
    7: "PANDORA_ERR_OUT_OF_MEMORY",
    8: "PANDORA_ERR_CUDA",
    9: "PANDORA_ERR_WORKSPACE_TOO_SMALL",
    10: "PANDORA_ERR_SIZE_LIMIT",
    11: "PANDORA_ERR_BAD_WEIGHT",
    12: "PANDORA_ERR_NOT_A_DENDROGRAM",
    13: "PANDORA_ERR_BAD_POINT",
}

FLAT_MAX_VERTICES = 536870912   # PANDORA_FLAT_MAX_VERTICES

SMALL_CAP = 4096          # largest tree the single-block solver takes
SMALL_BUCKETS = 13        # bucket k: trees with 2^k <= m < 2^(k+1) edges (k = 0 also m = 0)


class PandoraError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        self.name = STATUS_NAMES.get(self.code, "UNKNOWN")
        super().__init__(f"{what}: {self.name} ({self.code})" if what else self.name)


class Stats(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("level_edges", ctypes.c_int64 * MAX_LEVELS),
                ("level_vertices", ctypes.c_int64 * MAX_LEVELS)]


class Profile(ctypes.Structure):
    _fields_ = [("n_kernels", ctypes.c_int32), ("timing", ctypes.c_int32),
                ("name", (ctypes.c_char * 32) * 16), ("launches", ctypes.c_int64 * 16),
                ("elements", ctypes.c_int64 * 16), ("total_ms", ctypes.c_double * 16),
                ("kernels", ctypes.c_int64 * 16)]


class Tuning(ctypes.Structure):
    _fields_ = [("small_max_edges", ctypes.c_int32),
                ("small_threads", ctypes.c_int32 * SMALL_BUCKETS),
                ("split_min_permille", ctypes.c_int32)]


def library_path() -> str:
    return os.environ.get("PANDORA_LIBRARY") or os.path.join(HERE, _LIB_NAME)


def load_library():
    """Load libpandora.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "paper_2401_06089_gb300.build.build()")
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        SZ = ctypes.c_size_t
        lib.pandora_dendrogram.argtypes = [P, P, P, I64, P, P, P]
        lib.pandora_dendrogram_ws.argtypes = [P, P, P, I64, P, P, P, SZ, P, P]
        lib.pandora_dendrogram_host.argtypes = [P, P, P, I64, P, P, P]
        lib.pandora_dendrogram_batched.argtypes = [P, P, P, P, I64, I64, P, P, P]
        lib.pandora_dendrogram_batched_ws.argtypes = [P, P, P, P, I64, I64, P, P, P, SZ, P, P]
        lib.pandora_workspace_size.argtypes = [I64, I64, ctypes.POINTER(SZ)]
        lib.pandora_status_string.argtypes = [ctypes.c_int]
        lib.pandora_status_string.restype = ctypes.c_char_p
        lib.pandora_version.argtypes = []
        lib.pandora_dendrogram_async.argtypes = [P, P, P, I64, P, P, P, SZ, P]
        lib.pandora_dendrogram_batched_async.argtypes = [P, P, P, P, I64, I64, P, P, P, SZ, P]
        lib.pandora_dendrogram_batched_planned.argtypes = [P, P, P, P, P, I64, I64, P, P, P, SZ,
                                                           P]
        lib.pandora_workspace_status.argtypes = [P, P]
        lib.pandora_profile_start.argtypes = [ctypes.c_int]
        lib.pandora_profile_read.argtypes = [P]
        lib.pandora_set_tuning.argtypes = [P]
        lib.pandora_get_tuning.argtypes = [P]
        lib.pandora_hdbscan_labels.argtypes = [P, P, P, I64, ctypes.c_int32, P, P,
                                               ctypes.POINTER(I64), P]
        lib.pandora_membench.argtypes = [ctypes.c_int, P, P, P, I64, I64, I64, ctypes.c_uint64,
                                         ctypes.c_int, P]
        lib.pandora_mr_emst.argtypes = [P, I64, ctypes.c_int32, P, P, P, P, P]
        lib.pandora_set_wait_report_limit.argtypes = [I64]
        lib.pandora_sort_pairs_workspace_size.argtypes = [I64, ctypes.c_int32, ctypes.POINTER(SZ)]
        lib.pandora_sort_pairs.argtypes = [P, P, I64, ctypes.c_int32, P, P, P, SZ, P]
        for name in ("pandora_dendrogram", "pandora_dendrogram_ws", "pandora_dendrogram_batched",
                     "pandora_dendrogram_batched_ws", "pandora_workspace_size",
                     "pandora_version", "pandora_profile_start", "pandora_profile_read",
                     "pandora_dendrogram_async", "pandora_dendrogram_batched_async",
                     "pandora_workspace_status", "pandora_set_tuning", "pandora_get_tuning",
                     "pandora_dendrogram_batched_planned", "pandora_dendrogram_host",
                     "pandora_hdbscan_labels", "pandora_membench", "pandora_mr_emst",
                     "pandora_set_wait_report_limit", "pandora_sort_pairs_workspace_size",
                     "pandora_sort_pairs"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    _apply_default_tuning()
    return lib


TUNING_FILE = os.path.join(HERE, "tuning_gb300.json")


def _apply_default_tuning():
    """Apply the autotuner's file shipped beside the package (or the file named
    by PANDORA_TUNING; PANDORA_TUNING=none keeps the library defaults)."""
    path = os.environ.get("PANDORA_TUNING", TUNING_FILE)
    if path.lower() == "none" or not os.path.exists(path):
        return
    load_tuning(path)


def status_string(code: int) -> str:
    return load_library().pandora_status_string(int(code)).decode()


def workspace_size(total_edges: int, n_trees: int = 1) -> int:
    out = ctypes.c_size_t(0)
    st = load_library().pandora_workspace_size(int(total_edges), int(n_trees), ctypes.byref(out))
    if st:
        raise PandoraError(st, "pandora_workspace_size")
    return int(out.value)


def get_tuning() -> dict:
    """The process-wide small-tree settings: {"small_max_edges", "small_threads"}."""
    t = Tuning()
    st = load_library().pandora_get_tuning(ctypes.byref(t))
    if st:
        raise PandoraError(st, "pandora_get_tuning")
    return {"small_max_edges": int(t.small_max_edges),
            "small_threads": [int(x) for x in t.small_threads],
            "split_min_permille": int(t.split_min_permille)}


def set_tuning(small_max_edges: int | None = None, small_threads=None,
               split_min_permille: int | None = None) -> dict:
    """Change the small-tree settings (unspecified fields keep their value).

    ``small_max_edges`` is the largest tree (in edges) the single-block solver
    takes (0 turns it off, at most ``SMALL_CAP``); ``small_threads`` is a list
    of 13 block sizes (256, 512 or 1024), one per size bucket;
    ``split_min_permille`` is the share of a batch's edges (per mille) its
    small trees must hold before a batched call is split.  Returns the
    settings now in force."""
    cur = get_tuning()
    t = Tuning()
    t.small_max_edges = int(cur["small_max_edges"] if small_max_edges is None else small_max_edges)
    thr = cur["small_threads"] if small_threads is None else list(small_threads)
    if len(thr) != SMALL_BUCKETS:
        raise ValueError(f"small_threads needs {SMALL_BUCKETS} entries")
    for k, x in enumerate(thr):
        t.small_threads[k] = int(x)
    t.split_min_permille = int(cur["split_min_permille"] if split_min_permille is None
                               else split_min_permille)
    st = load_library().pandora_set_tuning(ctypes.byref(t))
    if st:
        raise PandoraError(st, "pandora_set_tuning")
    return get_tuning()


def load_tuning(path: str) -> dict:
    """Apply a tuning file written by ``paper_2401_06089_gb300.autotune``."""
    import json
    with open(path) as f:
        cfg = json.load(f)
    return set_tuning(cfg.get("small_max_edges"), cfg.get("small_threads"),
                      cfg.get("split_min_permille"))


def profile_start(timing: bool = False) -> None:
    """Reset the per-kernel counters; with ``timing`` also time every launch."""
    load_library().pandora_profile_start(1 if timing else 0)


def profile_read() -> dict:
    """{step: {"launches", "kernels", "elements", "ms"}} since the last
    profile_start ("launches" counts steps of the path, "kernels" the CUDA
    kernels they launched)."""
    pr = Profile()
    load_library().pandora_profile_read(ctypes.byref(pr))
    out = {}
    for k in range(pr.n_kernels):
        name = pr.name[k].value.decode()
        out[name] = {"launches": int(pr.launches[k]), "kernels": int(pr.kernels[k]),
                     "elements": int(pr.elements[k]),
                     "ms": float(pr.total_ms[k]) if pr.timing else None}
    return out


def _torch():
    import torch
    return torch


def _check(t, dtype, name, device=None, length=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (there is no CPU path)")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if t.dim() != 1 or not t.is_contiguous():
        raise ValueError(f"{name} must be 1-D and contiguous")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if length is not None and t.numel() != length:
        raise ValueError(f"{name} has {t.numel()} elements, expected {length}")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def _stats_dict(st: Stats):
    n = int(st.n_levels)
    return {"n_levels": n, "level_edges": [int(x) for x in st.level_edges[:n]],
            "level_vertices": [int(x) for x in st.level_vertices[:n]]}


def dendrogram(u, v, w, *, workspace=None, stats: bool = False, out=None):
    """Single-linkage dendrogram of one tree (``pandora_dendrogram``).

    u, v: int32 CUDA tensors [m] (vertex ids in [0, m]); w: float32 [m].
    Returns (edge_parent int32[m], vertex_parent int32[m+1]) on the same
    device, plus a statistics dict when ``stats`` is True.  ``workspace`` (a
    uint8 CUDA tensor of at least ``workspace_size(m)`` bytes) avoids the
    library's own stream-ordered allocation.  ``out`` = (edge_parent,
    vertex_parent) reuses output tensors.
    """
    torch = _torch()
    lib = load_library()
    _check(w, torch.float32, "w")
    dev = w.device
    m = w.numel()
    _check(u, torch.int32, "u", dev, m)
    _check(v, torch.int32, "v", dev, m)
    if out is None:
        ep = torch.empty(m, dtype=torch.int32, device=dev)
        vp = torch.empty(m + 1, dtype=torch.int32, device=dev)
    else:
        ep, vp = out
        _check(ep, torch.int32, "edge_parent", dev, m)
        _check(vp, torch.int32, "vertex_parent", dev, m + 1)
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st_out = Stats()
        if workspace is None and not stats:
            st = lib.pandora_dendrogram(_ptr(u), _ptr(v), _ptr(w), m, _ptr(ep), _ptr(vp), stream)
        else:
            if workspace is None:
                workspace = torch.empty(workspace_size(m, 1), dtype=torch.uint8, device=dev)
            st = lib.pandora_dendrogram_ws(_ptr(u), _ptr(v), _ptr(w), m, _ptr(ep), _ptr(vp),
                                           _ptr(workspace), workspace.numel(),
                                           ctypes.byref(st_out), stream)
    if st:
        raise PandoraError(st, "pandora_dendrogram")
    if stats:
        return ep, vp, _stats_dict(st_out)
    return ep, vp


def hdbscan_labels(edge_parent, vertex_parent, w, min_cluster_size: int, *,
                   stability: bool = False):
    """HDBSCAN* flat clusters of a dendrogram (``pandora_hdbscan_labels``).

    ``edge_parent`` (int32[m]), ``vertex_parent`` (int32[m + 1]) and ``w``
    (float32[m], positive) are CUDA tensors, e.g. the outputs of
    ``dendrogram`` and its weights.  Returns int32 labels (-1 = noise,
    clusters numbered by their smallest point id); with ``stability`` also
    the float64 stability of every cluster, indexed by label.
    """
    torch = _torch()
    lib = load_library()
    _check(vertex_parent, torch.int32, "vertex_parent")
    dev = vertex_parent.device
    n = vertex_parent.numel()
    m = max(n - 1, 0)
    _check(edge_parent, torch.int32, "edge_parent", dev, m)
    _check(w, torch.float32, "w", dev, m)
    mcs = int(min_cluster_size)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    stab = None
    if stability:
        stab = torch.empty(max(n // max(mcs, 1), 1), dtype=torch.float64, device=dev)
    nc = ctypes.c_int64(0)
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st = lib.pandora_hdbscan_labels(_ptr(edge_parent), _ptr(vertex_parent), _ptr(w), n, mcs,
                                        _ptr(labels), _ptr(stab) if stability else None,
                                        ctypes.byref(nc), stream)
    if st:
        raise PandoraError(st, "pandora_hdbscan_labels")
    if stability:
        return labels, stab[: nc.value]
    return labels


def dendrogram_host(u, v, w, *, out=None, device=None):
    """``pandora_dendrogram_host``: CPU tensors in (pinned copies fastest),
    CPU tensors out; the library moves the data and overlaps the copies with
    the path.  ``device``: the CUDA device to run on (default: current)."""
    torch = _torch()
    lib = load_library()
    m = w.numel()
    for t, dt, name in ((u, torch.int32, "u"), (v, torch.int32, "v"), (w, torch.float32, "w")):
        if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous() or t.numel() != m:
            raise ValueError(f"{name} must be a contiguous CPU {dt} tensor of {m} elements")
    if out is None:
        pin = u.is_pinned()
        ep = torch.empty(m, dtype=torch.int32, pin_memory=pin)
        vp = torch.empty(m + 1, dtype=torch.int32, pin_memory=pin)
    else:
        ep, vp = out
        for t, n, name in ((ep, m, "edge_parent"), (vp, m + 1, "vertex_parent")):
            if t.device.type != "cpu" or t.dtype != torch.int32 or not t.is_contiguous() \
                    or t.numel() != n:
                raise ValueError(f"{name} must be a contiguous CPU int32 tensor of {n} elements")
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st = lib.pandora_dendrogram_host(u.data_ptr(), v.data_ptr(), w.data_ptr(), m,
                                         ep.data_ptr(), vp.data_ptr(), stream)
    if st:
        raise PandoraError(st, "pandora_dendrogram_host")
    return ep, vp


def dendrogram_batched(u, v, w, edge_offsets, *, workspace=None, stats: bool = False, out=None):
    """Dendrograms of many trees packed by ``edge_offsets`` (int64, CUDA).

    Tree t owns edges [off[t], off[t+1]) and vertices [off[t]+t, off[t+1]+t+1)
    of the packed arrays; ids in u, v and in the outputs are tree-local.
    Returns (edge_parent int32[M], vertex_parent int32[M + T]).
    """
    torch = _torch()
    lib = load_library()
    _check(w, torch.float32, "w")
    dev = w.device
    m = w.numel()
    _check(u, torch.int32, "u", dev, m)
    _check(v, torch.int32, "v", dev, m)
    _check(edge_offsets, torch.int64, "edge_offsets", dev)
    n_trees = edge_offsets.numel() - 1
    if n_trees < 0:
        raise ValueError("edge_offsets needs n_trees + 1 entries")
    if out is None:
        ep = torch.empty(m, dtype=torch.int32, device=dev)
        vp = torch.empty(m + n_trees, dtype=torch.int32, device=dev)
    else:
        ep, vp = out
        _check(ep, torch.int32, "edge_parent", dev, m)
        _check(vp, torch.int32, "vertex_parent", dev, m + n_trees)
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st_out = Stats()
        if workspace is None and not stats:
            st = lib.pandora_dendrogram_batched(_ptr(u), _ptr(v), _ptr(w), _ptr(edge_offsets),
                                                n_trees, m, _ptr(ep), _ptr(vp), stream)
        else:
            if workspace is None:
                workspace = torch.empty(workspace_size(m, max(n_trees, 1)), dtype=torch.uint8,
                                        device=dev)
            st = lib.pandora_dendrogram_batched_ws(_ptr(u), _ptr(v), _ptr(w), _ptr(edge_offsets),
                                                   n_trees, m, _ptr(ep), _ptr(vp),
                                                   _ptr(workspace), workspace.numel(),
                                                   ctypes.byref(st_out), stream)
    if st:
        raise PandoraError(st, "pandora_dendrogram_batched")
    if stats:
        return ep, vp, _stats_dict(st_out)
    return ep, vp


def dendrogram_async(u, v, w, workspace, out):
    """Enqueue ``pandora_dendrogram_async`` on the current stream and return.

    Nothing is synchronised or allocated, so the call can be captured in a
    CUDA graph.  ``out`` = (edge_parent, vertex_parent) receives the result
    once the stream reaches it; device-detected errors are read with
    ``workspace_status(workspace)``.
    """
    torch = _torch()
    lib = load_library()
    _check(w, torch.float32, "w")
    dev = w.device
    m = w.numel()
    _check(u, torch.int32, "u", dev, m)
    _check(v, torch.int32, "v", dev, m)
    ep, vp = out
    _check(ep, torch.int32, "edge_parent", dev, m)
    _check(vp, torch.int32, "vertex_parent", dev, m + 1)
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st = lib.pandora_dendrogram_async(_ptr(u), _ptr(v), _ptr(w), m, _ptr(ep), _ptr(vp),
                                          _ptr(workspace), workspace.numel(), stream)
    if st:
        raise PandoraError(st, "pandora_dendrogram_async")


def dendrogram_batched_async(u, v, w, edge_offsets, workspace, out):
    """Enqueue ``pandora_dendrogram_batched_async`` (see ``dendrogram_async``)."""
    torch = _torch()
    lib = load_library()
    _check(w, torch.float32, "w")
    dev = w.device
    m = w.numel()
    _check(u, torch.int32, "u", dev, m)
    _check(v, torch.int32, "v", dev, m)
    _check(edge_offsets, torch.int64, "edge_offsets", dev)
    n_trees = edge_offsets.numel() - 1
    ep, vp = out
    _check(ep, torch.int32, "edge_parent", dev, m)
    _check(vp, torch.int32, "vertex_parent", dev, m + n_trees)
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st = lib.pandora_dendrogram_batched_async(_ptr(u), _ptr(v), _ptr(w), _ptr(edge_offsets),
                                                  n_trees, m, _ptr(ep), _ptr(vp),
                                                  _ptr(workspace), workspace.numel(), stream)
    if st:
        raise PandoraError(st, "pandora_dendrogram_batched_async")


def dendrogram_batched_planned(u, v, w, edge_offsets, host_edge_offsets, workspace, out):
    """Enqueue ``pandora_dendrogram_batched_planned``: like
    ``dendrogram_batched_async`` plus a host copy of the offsets (a CPU int64
    tensor, numpy array or list with the same values), which lets small trees
    take the single-block solver without a host synchronisation."""
    import numpy as np
    torch = _torch()
    lib = load_library()
    _check(w, torch.float32, "w")
    dev = w.device
    m = w.numel()
    _check(u, torch.int32, "u", dev, m)
    _check(v, torch.int32, "v", dev, m)
    _check(edge_offsets, torch.int64, "edge_offsets", dev)
    n_trees = edge_offsets.numel() - 1
    h = np.ascontiguousarray(np.asarray(host_edge_offsets, dtype=np.int64))
    if h.shape != (n_trees + 1,):
        raise ValueError("host_edge_offsets must have n_trees + 1 entries")
    ep, vp = out
    _check(ep, torch.int32, "edge_parent", dev, m)
    _check(vp, torch.int32, "vertex_parent", dev, m + n_trees)
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st = lib.pandora_dendrogram_batched_planned(
            _ptr(u), _ptr(v), _ptr(w), _ptr(edge_offsets), h.ctypes.data, n_trees, m, _ptr(ep),
            _ptr(vp), _ptr(workspace), workspace.numel(), stream)
    if st:
        raise PandoraError(st, "pandora_dendrogram_batched_planned")


def workspace_status(workspace, raise_on_error: bool = True) -> int:
    """Wait for the current stream and return the workspace's device status."""
    torch = _torch()
    lib = load_library()
    dev = workspace.device
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st = lib.pandora_workspace_status(_ptr(workspace), stream)
    if st and raise_on_error:
        raise PandoraError(st, "device status")
    return st


MEMBENCH_KINDS = {"gather32": 0, "gather64": 1, "scatter32": 2, "scatter64": 3,
                  "atomicmin64": 4, "copy32": 5}


def membench(kind: str, buf, *, n_access: int, window: int = 0, seed: int = 0,
             blocks_per_sm: int = 8, dst=None, sink=None) -> None:
    """Enqueue one random-access micro-benchmark kernel (``pandora_membench``)
    on the current stream: ``n_access`` accesses of ``kind`` to ``buf`` (a
    CUDA tensor of 4- or 8-byte elements) at hashed positions; the caller
    times it with CUDA events."""
    torch = _torch()
    if kind not in MEMBENCH_KINDS:
        raise ValueError(f"unknown kind {kind!r}")
    if not (isinstance(buf, torch.Tensor) and buf.is_cuda and buf.is_contiguous()):
        raise ValueError("buf must be a contiguous CUDA tensor")
    width = 8 if kind.endswith("64") else 4
    if buf.element_size() != width:
        raise TypeError(f"{kind} needs {width}-byte elements")
    if sink is None:
        sink = torch.zeros(1, dtype=torch.int32, device=buf.device)
    lib = load_library()
    stream = ctypes.c_void_p(torch.cuda.current_stream(buf.device).cuda_stream)
    st = lib.pandora_membench(MEMBENCH_KINDS[kind], _ptr(buf), _ptr(dst), _ptr(sink),
                              buf.numel(), int(n_access), int(window), int(seed),
                              int(blocks_per_sm), stream)
    if st:
        raise PandoraError(st, "pandora_membench")


EMST_MAX_MIN_PTS = 32   # PANDORA_EMST_MAX_MIN_PTS


def mr_emst(points, min_pts: int, *, core: bool = False):
    """Mutual-reachability minimum spanning tree of 3-D points
    (``pandora_mr_emst``): points is a float32 CUDA tensor [n, 3]; returns
    int32 u, v and float32 w of the n - 1 tree edges (u < v), and with
    ``core`` also the float32 squared core distance of every point."""
    torch = _torch()
    if not isinstance(points, torch.Tensor) or not points.is_cuda:
        raise ValueError("points must be a CUDA tensor (there is no CPU path)")
    if points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 3 or \
            not points.is_contiguous():
        raise ValueError("points must be a contiguous float32 tensor of shape [n, 3]")
    n = points.shape[0]
    dev = points.device
    u = torch.empty(max(n - 1, 0), dtype=torch.int32, device=dev)
    v = torch.empty(max(n - 1, 0), dtype=torch.int32, device=dev)
    w = torch.empty(max(n - 1, 0), dtype=torch.float32, device=dev)
    cs = torch.empty(n, dtype=torch.float32, device=dev) if core else None
    lib = load_library()
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st = lib.pandora_mr_emst(_ptr(points), n, int(min_pts), _ptr(u), _ptr(v), _ptr(w),
                                 _ptr(cs), stream)
    if st:
        raise PandoraError(st, "pandora_mr_emst")
    return (u, v, w, cs) if core else (u, v, w)


def sort_pairs(keys, vals, key_bits: int = 32):
    """Stable radix sort of (key, value) pairs by key (``pandora_sort_pairs``,
    the sort of the dendrogram's weight and chain-key steps): keys and vals
    are contiguous 4-byte CUDA tensors of equal length, every key below
    2^key_bits; returns new (keys, vals) tensors in key order, equal keys in
    input order.  Synchronises the current stream."""
    torch = _torch()
    for name, t in (("keys", keys), ("vals", vals)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()
                and t.element_size() == 4):
            raise ValueError(f"{name} must be a contiguous CUDA tensor of 4-byte elements")
    if keys.numel() != vals.numel():
        raise ValueError("keys and vals differ in length")
    n = keys.numel()
    dev = keys.device
    lib = load_library()
    need = ctypes.c_size_t()
    st = lib.pandora_sort_pairs_workspace_size(n, int(key_bits), ctypes.byref(need))
    if st:
        raise PandoraError(st, "pandora_sort_pairs_workspace_size")
    ws = torch.empty(max(need.value, 16), dtype=torch.uint8, device=dev)
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    with torch.cuda.device(dev):
        stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        st = lib.pandora_sort_pairs(_ptr(keys), _ptr(vals), n, int(key_bits), _ptr(ko), _ptr(vo),
                                    _ptr(ws), ws.numel(), stream)
    if st:
        raise PandoraError(st, "pandora_sort_pairs")
    return ko, vo


def set_wait_report_limit(spins: int) -> None:
    """Make the bounded device loops (look-back waits, union-find loops)
    report PANDORA_ERR_ITERATION_LIMIT once they run longer than ``spins``
    iterations, without cutting them short (``pandora_set_wait_report_limit``;
    negative: the default)."""
    load_library().pandora_set_wait_report_limit(int(spins))
