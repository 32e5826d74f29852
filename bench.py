#!/usr/bin/env python
"""Benchmark: MST edges/s to single-linkage dendrogram on GB300.

Default workload: a random recursive tree of n = 10^8 vertices (m = 10^8 - 1
edges) with uniform fp32 weights k * 2**-24, seed 1; the 10^8-vertex skewed
path (w_i = fp32(i + U(0, 0.5))) is timed the same way and reported beside
it.  One step = one full dendrogram (sort, every contraction level,
expansion, chain sort, link) through the library's C ABI with the inputs
resident in HBM; ``e2e`` repeats the step through ``pandora_dendrogram_host``
with pinned host buffers (H2D of u, v, w and D2H of both outputs inside the
timed region, overlapped with the path by the library).

``--impl reference`` times the CPU oracle (plain C Kruskal, one thread) on a
bounded sample of the same workload instead.

Prints ONE JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MST edges/s to dendrogram on 1 GB300 + HBM roofline %; batched vs per-tree speedup"
# vertices of the tree the reference arm (the CPU oracle) times per step
REFERENCE_SAMPLE = 10_000_000
UNIT = "edges/s"
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    "rrt_1e8": dict(family="rrt", n=10**8, seed=1,
                    desc="random recursive tree, uniform fp32 weights k*2^-24"),
    "path_1e8": dict(family="path_skewed", n=10**8, seed=2,
                     desc="skewed path, w_i = fp32(i + U(0,0.5))"),
    "rrt_1e4": dict(family="rrt", n=10**4, seed=0,
                    desc="random recursive tree, uniform fp32 weights k*2^-24"),
    "serving": dict(family="serving", n=2000, seed=5,
                    desc="Poisson arrivals of random recursive trees, vertex counts "
                         "log-uniform in [1e3, 1e7], uniform fp32 weights"),
    "hdbscan_4m": dict(family="hdbscan", n=4_000_000, seed=3,
                       desc="mutual-reachability spanning tree (minPts 16) of 4e6 3-D points "
                            "from a 32-component Gaussian mixture"),
    "batched_4096": dict(family="batch", n=4096, seed=4,
                         desc="4096 trees, vertex counts log-uniform in [1e2, 1e6], "
                              "random recursive or skewed path by a fair coin"),
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="rrt_1e8")
    ap.add_argument("--n", type=int, default=None, help="override the vertex count")
    ap.add_argument("--no-extra", action="store_true", help="skip the path family line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--check", action="store_true",
                    help="check the structure of the outputs after the timed region (one root, "
                         "edge order, two children per edge, Eq. 1)")
    ap.add_argument("--async-api", action="store_true",
                    help="time pandora_dendrogram_async (worst-case level count, no host sync)")
    ap.add_argument("--membench", action="store_true",
                    help="only measure the random-access ceilings (pandora_membench) and print "
                         "them as one JSON line")
    ap.add_argument("--emst", type=int, default=0, metavar="POINTS",
                    help="only time the mutual-reachability spanning tree (pandora_mr_emst) of "
                         "this many Gaussian-mixture points and print one JSON line")
    ap.add_argument("--membench-bps", type=int, nargs="*", default=[4, 8, 16],
                    help="blocks per SM of the --membench kernels")
    ap.add_argument("--membench-reps", type=int, default=5)
    ap.add_argument("--flat", type=int, default=0, metavar="MCS",
                    help="also time HDBSCAN* flat clusters (pandora_hdbscan_labels) with this "
                         "min_cluster_size on the workload's dendrogram")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def make_tree(spec, n=None):
    from paper_2401_06089_gb300 import inputs
    n = n or spec["n"]
    if spec["family"] == "rrt":
        return inputs.rrt(n, spec["seed"])
    if spec["family"] == "hdbscan":
        return inputs.hdbscan_tree(n, spec["seed"])
    return inputs.path_skewed(n, spec["seed"])


def dendrogram_structure(u, v, w, ep, vp):
    """Checks of a dendrogram that need no reference result (numpy, host): one
    root; every edge later than its children in the total order of Section 3.1
    (weight, -0.0 before +0.0, index); two children per edge; every vertex's
    parent is its lightest incident edge (Eq. 1).  Necessary conditions only:
    element-by-element parity with the oracle is the test suite's job."""
    import numpy as np
    m = len(w)
    n = m + 1
    out = {"edges": int(m)}
    if m == 0:
        out["ok"] = bool(len(vp) == 1 and vp[0] == -1)
        return out
    w = np.asarray(w, np.float32)
    order = np.lexsort((np.arange(m), ~np.signbit(w), w))   # ascending total order
    rank = np.empty(m, np.int64)
    rank[order] = np.arange(m)
    ep = np.asarray(ep, np.int64)
    vp = np.asarray(vp, np.int64)
    roots = int((ep == -1).sum())
    inner = ep >= 0
    in_range = bool(((ep >= -1) & (ep < m)).all() and ((vp >= 0) & (vp < m)).all())
    out["one_root"] = roots == 1
    out["parents_in_range"] = in_range
    if not in_range:
        out["ok"] = False
        return out
    out["parent_later_in_order"] = bool((rank[ep[inner]] > rank[inner.nonzero()[0]]).all())
    kids = np.bincount(ep[inner], minlength=m) + np.bincount(vp, minlength=m)
    out["two_children_each"] = bool((kids == 2).all())
    lightest = np.full(n, np.iinfo(np.int64).max)
    np.minimum.at(lightest, np.asarray(u, np.int64), rank)
    np.minimum.at(lightest, np.asarray(v, np.int64), rank)
    out["vertex_parent_lightest"] = bool((rank[vp] == lightest).all())
    out["ok"] = bool(out["one_root"] and out["parent_later_in_order"] and
                     out["two_children_each"] and out["vertex_parent_lightest"])
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) kept only inside [t_start, t_stop]."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        self.lines = []
        self.t_start = self.t_stop = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def start(self):
        self.t_start = time.time()

    def stop(self):
        self.t_stop = time.time()
        time.sleep(0.25)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.t_start is not None and not (self.t_start - 0.2 <= t <= self.t_stop + 0.2):
                continue
            rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        for r in rows:
            for name, col in (("hw_slowdown", 5), ("hw_thermal_slowdown", 6),
                              ("sw_thermal_slowdown", 7), ("sw_power_cap", 8)):
                if r[col].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ---- algorithmic bytes per kernel: each element touch counted once, a random
# 4-byte access as 4 bytes (the roofline numerator) ---------------------------
def sort_weight_bytes(m, launches):
    """Bytes of the (weight, index) sort passes, which carry the endpoints:
    first pass 28 B/edge (read w, u, v; write key, index, u, v), middle 32
    (read and write 16), last 28 (read 16; write index 4 and (u, v) 8); a
    single pass 24."""
    if launches == 0:
        return 0
    if launches == 1:
        return 24 * m
    return (28 + 32 * (launches - 2) + 28) * m


# per element of the kernel's launch size (edges or vertices of the level)
MODEL_BYTES = {"hist_weights": 4, "onesweep_chains": 16, "init_level": 8, "mark": 24,
               "tail_levels": 25,
               "ptr_init": 28, "compress": 16, "compact": 35, "expand": 25, "link": 16,
               "check_offsets": 16, "fill": 4}


# Level 0 of a tree above 2^24 vertices marks by buckets with the Eq. 2 flag
# pass: mark then also reads the caller ids (4 B per edge) and writes
# vertex_parent (4 B per vertex) and the flags (2 bits per edge); ptr_init
# reads only the vertex's own word and its edge's flags (8 + 1/4 B) and writes
# the pointer (4 B); root finding reads and tags the pointer words (own word
# read and written, at least one pointer target read: 12 B); compact (see
# compact_level0_bytes) reads the pointer tag of one endpoint of a contracted
# edge and of both endpoints of an alpha-edge.
FLAGGED_LEVEL0_MIN_VERTICES = (1 << 24) + 1
LEVEL0_FLAGGED_BYTES = {"mark": 32.25, "ptr_init": 12.25, "compress": 12}


def compact_level0_bytes(m, m1):
    """Flagged level-0 compact of m edges of which m1 are alpha-edges: every
    edge reads its endpoints and flags (8 + 1/4 B); a contracted edge reads one
    4-byte tag and writes its level and supervertex (1 + 4 B); an alpha-edge
    reads two tags and writes its relabelled endpoints and rank (8 + 4 B)."""
    return m * 8.25 + (m - m1) * 9 + m1 * 20


def model_bytes(name, prof_entry, m, n_passes_w, level0_calls=0, m1=0):
    """Algorithmic bytes of all launches of `name`; `level0_calls` launches
    of the step ran a flagged level 0 of m edges with m1 alpha-edges (see
    above)."""
    e = prof_entry["elements"]
    if name == "onesweep_weights":
        return sort_weight_bytes(m, n_passes_w) * (prof_entry["launches"] // max(n_passes_w, 1))
    if name == "compact" and level0_calls:
        return (compact_level0_bytes(m, m1) * level0_calls +
                MODEL_BYTES[name] * (e - m * level0_calls))
    if name in LEVEL0_FLAGGED_BYTES and level0_calls:
        n0 = m if name == "mark" else m + 1
        return (LEVEL0_FLAGGED_BYTES[name] * n0 * level0_calls +
                MODEL_BYTES[name] * (e - n0 * level0_calls))
    return MODEL_BYTES.get(name, 0) * e


def dendrogram_height(edge_parent, vertex_parent):
    """Height of a dendrogram (Section 3.1, skewness): the most edge nodes on
    a path from the root edge down to a vertex.  Depths of the edges by
    pointer jumping on edge_parent (torch, on the tensors' device: a
    measurement of the output, not part of the timed path); a vertex sits one
    below its parent edge."""
    import torch
    ep = edge_parent.to(torch.int64)
    m = ep.numel()
    if m == 0:
        return 0
    idx = torch.arange(m, device=ep.device)
    root = ep < 0
    p = torch.where(root, idx, ep)
    d = (~root).to(torch.int64)            # edges between i and p[i]
    for _ in range(64):
        pp = p[p]
        if torch.equal(pp, p):
            break
        d = d + d[p]
        p = pp
    vp = vertex_parent.to(torch.int64)
    return int((d[vp[vp >= 0]] + 1).max().item())


def skewness(edge_parent, vertex_parent):
    """{height, ideal = log2 n, ratio}: the paper's skewness measure."""
    import math
    n = vertex_parent.numel()
    h = dendrogram_height(edge_parent, vertex_parent)
    ideal = math.log2(n) if n > 1 else 1.0
    return {"height": h, "ideal_log2_n": round(ideal, 3), "ratio": round(h / ideal, 2)}


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary of `kernel`, or None
    when the kernel's source changed since the counters were taken."""
    summary = os.path.join(ROOT, "profiles", f"{kernel}.md")
    if not os.path.exists(summary):
        return None
    text = open(summary).read()
    m1 = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    m2 = re.search(r"source_sha256:\s*([0-9a-f]+)", text)
    m3 = re.search(r"source_file:\s*(\S+)", text)
    if not (m1 and m2 and m3):
        return None
    src = os.path.join(ROOT, m3.group(1))
    if not os.path.exists(src):
        return None
    if hashlib.sha256(open(src, "rb").read()).hexdigest() != m2.group(1):
        return None
    return float(m1.group(1))


KERNEL_SOURCES = {"onesweep_weights": "sort", "onesweep_chains": "sort", "hist_weights": "sort",
                  "mark": "levels", "ptr_init": "levels", "compress": "levels",
                  "compact": "levels", "expand": "expand", "link": "expand"}


# ---------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args):
    """The CPU oracle (the reference arm of this benchmark: the paper ships no
    code) on a bounded sample of the workload, rank 0 only.  Every step is one
    oracle dendrogram of the same sample in the all-core mode (edge sort on
    every host core, union-find on one), the setting of the paper's UnionFind
    baseline (parallel sort, sequential union-find).  The sample, not the full
    workload, is what the line's config names."""
    import oracle
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    spec = WORKLOADS[args.workload]
    n_full = args.n or spec["n"]
    n_sample = min(n_full, REFERENCE_SAMPLE)
    t = make_tree(spec, n_sample)
    oracle.build()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.dendrogram_threads(t.u, t.v, t.w, cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.dendrogram_threads(t.u, t.v, t.w, cores)
        times.append(time.perf_counter() - t0)
    sec = sum(times) / len(times)
    value = t.m / sec
    sample = (f"{spec['family']} n={n_sample} seed={spec['seed']} (same generator), edge sort "
              f"on {cores} threads, union-find on one")
    config = config_of(args, spec)
    if n_sample != n_full:
        config["workload"] = f"{config['workload']}_sample_n{n_sample}"
        config["n_vertices"] = n_sample
        config["n_edges"] = n_sample - 1
        config["sample_of"] = f"{args.workload} (n={n_full})"
        config["l2"] = "host caches; the oracle runs on the CPU"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def measure_rrt_1e4(pd, torch, args, reps=200):
    """Configuration rrt_1e4 (n = 10^4, seed 0): launch-bound; the blocking
    call by wall clock, the asynchronous call and its CUDA-graph replay by
    CUDA events on the launching stream."""
    spec = WORKLOADS["rrt_1e4"]
    t = make_tree(spec)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    u = torch.from_numpy(t.u).to(dev)
    v = torch.from_numpy(t.v).to(dev)
    w = torch.from_numpy(t.w).to(dev)
    ws = torch.empty(pd.workspace_size(t.m), dtype=torch.uint8, device=dev)
    ep = torch.empty(t.m, dtype=torch.int32, device=dev)
    vp = torch.empty(t.m + 1, dtype=torch.int32, device=dev)
    for _ in range(10):
        pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
    torch.cuda.synchronize()
    blocking_ms = (time.perf_counter() - t0) * 1e3 / reps
    ref = (ep.clone(), vp.clone())
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    for _ in range(10):
        pd.dendrogram_async(u, v, w, ws, (ep, vp))
    a.record(stream)
    for _ in range(reps):
        pd.dendrogram_async(u, v, w, ws, (ep, vp))
    b.record(stream)
    b.synchronize()
    async_ms = a.elapsed_time(b) / reps
    pd.workspace_status(ws)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        pd.dendrogram_async(u, v, w, ws, (ep, vp))
    stream.wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        pd.dendrogram_async(u, v, w, ws, (ep, vp))
    for _ in range(10):
        g.replay()
    a.record(stream)
    for _ in range(reps):
        g.replay()
    b.record(stream)
    b.synchronize()
    graph_ms = a.elapsed_time(b) / reps
    pd.workspace_status(ws)
    same = bool(torch.equal(ep, ref[0]) and torch.equal(vp, ref[1]))
    return {"n_vertices": t.n, "seed": spec["seed"], "reps": reps,
            "blocking_ms": blocking_ms, "async_ms": async_ms, "graph_ms": graph_ms,
            "edges_per_s_blocking": t.m / (blocking_ms / 1e3),
            "edges_per_s_graph": t.m / (graph_ms / 1e3),
            "timing": "blocking: wall clock; async and graph: CUDA events on the stream",
            "outputs_equal_across_apis": same}


def summarize_batched(line):
    keep = ("value", "unit", "ms_per_step", "per_tree_blocking_ms", "per_tree_async_ms",
            "speedup_vs_per_tree_blocking", "speedup_vs_per_tree_async", "gpu_launches_per_step",
            "forest_async_graph_ms", "blocking_kernel_ms", "structure", "clocks")
    out = {k: line[k] for k in keep if k in line}
    out["config"] = {k: line["config"][k] for k in ("n_trees", "total_edges", "family", "mode")}
    kern = line.get("blocking_kernels", {})
    tot = sum((e["ms"] or 0.0) for e in kern.values()) or 1.0
    out["blocking_kernel_share"] = {k: round((e["ms"] or 0.0) / tot, 4) for k, e in kern.items()}
    return out


def summarize_serving(line):
    keep = ("value", "unit", "latency_ms", "saturated_edges_per_s",
            "per_request_blocking_edges_per_s", "speedup_saturated_vs_per_request",
            "max_batches_in_flight", "gpu_launches", "clocks")
    out = {k: line[k] for k in keep if k in line}
    out["config"] = line["config"]
    return out


def measure_hdbscan(pd, torch, args, n_points=None, reps=20, mcs=16):
    """Configuration hdbscan_4m end to end on the GPU: 4e6 points of the
    32-component Gaussian mixture, their exact mutual-reachability minimum
    spanning tree (minPts 16) by pandora_mr_emst, the dendrogram of that tree
    (timed like the headline) and its HDBSCAN* flat clusters."""
    import numpy as np
    from paper_2401_06089_gb300 import inputs
    spec = WORKLOADS["hdbscan_4m"]
    n = n_points or spec["n"]
    pts = torch.from_numpy(inputs.gmm_points(n, spec["seed"]).astype(np.float32)).cuda()
    dev = pts.device
    stream = torch.cuda.current_stream(dev)
    u, v, w = pd.mr_emst(pts, 16)   # warm-up
    torch.cuda.synchronize()
    emst_ms = []
    for _ in range(3):
        t0 = time.perf_counter()
        u, v, w = pd.mr_emst(pts, 16)
        torch.cuda.synchronize()
        emst_ms.append((time.perf_counter() - t0) * 1e3)
    m = u.numel()
    ws = torch.empty(pd.workspace_size(m), dtype=torch.uint8, device=dev)
    ep = torch.empty(m, dtype=torch.int32, device=dev)
    vp = torch.empty(m + 1, dtype=torch.int32, device=dev)
    for _ in range(3):
        pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
    b.record(stream)
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    labels = pd.hdbscan_labels(ep, vp, w, mcs)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(3):
        labels = pd.hdbscan_labels(ep, vp, w, mcs)
    b.record(stream)
    b.synchronize()
    flat_ms = a.elapsed_time(b) / 3
    lab = labels.cpu().numpy()
    st = dendrogram_structure(u.cpu().numpy(), v.cpu().numpy(), w.cpu().numpy(),
                              ep.cpu().numpy(), vp.cpu().numpy())
    emst = statistics.median(emst_ms)
    return {"value": m / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": reps,
            "n_points": n, "min_pts": 16, "seed": spec["seed"],
            "tree": "exact mutual-reachability minimum spanning tree (pandora_mr_emst, float32 "
                    "reading), computed on the GPU",
            "emst_ms": emst, "emst_points_per_s": n / (emst / 1e3),
            "emst_timing": "wall clock around the blocking call, median of 3",
            "emst_bound": EMST_BOUND,
            "flat_clusters": {"min_cluster_size": mcs, "ms_per_call": flat_ms,
                              "clusters": int(lab.max()) + 1,
                              "noise_fraction": float((lab < 0).mean())},
            "pipeline_ms": emst + ms + flat_ms,
            "skewness": skewness(ep, vp),
            "structure_ok": st["ok"]}


def cpu_baseline(spec, n_override=None, n_sample=10_000_000):
    """The CPU oracle on a bounded sample of the workload: one thread, and the
    all-core mode (sort on every host core, union-find sequential)."""
    import oracle
    oracle.build()
    n_s = min(n_override or spec["n"], n_sample)
    ts = make_tree(spec, n_s)
    t0 = time.perf_counter()
    oracle.dendrogram(ts.u, ts.v, ts.w)
    sec1 = time.perf_counter() - t0
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.dendrogram_threads(ts.u, ts.v, ts.w, cores)
    secn = time.perf_counter() - t0
    return {"value": ts.m / sec1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{spec['family']} n={n_s} seed={spec['seed']} (same generator), "
                      f"one thread, {sec1:.1f} s",
            "all_cores": {"value": ts.m / secn, "unit": UNIT, "cores": cores, "kind": "oracle",
                          "sample": f"same sample, sort on {cores} threads and union-find on "
                                    f"one, {secn:.1f} s"}}


def config_of(args, spec):
    n = args.n or spec["n"]
    return {"workload": f"{args.workload}" + (f"_n{n}" if args.n else ""), "n_vertices": n,
            "n_edges": n - 1, "family": spec["desc"], "seed": spec["seed"],
            "layout": "vertices relabelled, edges shuffled, orientations flipped at random",
            "l2": "inputs larger than L2 (12 B/edge in, 8 B/edge out)" if n > 20_000_000
            else "working set fits in L2",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


def time_device(pd, torch, t, steps, warmup, profile=True):
    dev = torch.device("cuda")
    u = torch.from_numpy(t.u).to(dev)
    v = torch.from_numpy(t.v).to(dev)
    w = torch.from_numpy(t.w).to(dev)
    ws = torch.empty(pd.workspace_size(t.m), dtype=torch.uint8, device=dev)
    ep = torch.empty(t.m, dtype=torch.int32, device=dev)
    vp = torch.empty(t.m + 1, dtype=torch.int32, device=dev)
    for _ in range(warmup):
        pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
    torch.cuda.synchronize()
    return dict(u=u, v=v, w=w, ws=ws, ep=ep, vp=vp)


def run_batched(args):
    world, rank, _ = dist_setup(args)
    line = measure_batched(args)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_batched(args, n_trees=None, init_dist=True):
    """Batched workload: the planned batched call captured in a CUDA graph,
    against one call per tree on the same GPU.  With N ranks the batch has
    N * n_trees trees, sharded by whole trees (largest first to the least
    loaded rank, no collective on the data path); each rank builds and solves
    only its shard, so the work per GPU stays fixed (weak scaling)."""
    import numpy as np
    import torch
    import paper_2401_06089_gb300 as pd
    from paper_2401_06089_gb300 import inputs
    world, rank, local = dist_setup(args)
    if world > 1 and init_dist:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif world > 1:
        import torch.distributed as dist
    else:
        dist = None
    spec = WORKLOADS["batched_4096"]
    n_trees = n_trees or args.n or spec["n"]
    n_total = n_trees * world
    if world > 1:
        from paper_2401_06089_gb300.sharding import shard_trees
        sizes = inputs.batch_sizes(n_total, 100, 1_000_000, spec["seed"])
        mine = shard_trees(sizes - 1, world)[rank]
        b = inputs.batch(n_total, 100, 1_000_000, seed=spec["seed"], only=mine)
    else:
        b = inputs.batch(n_trees, 100, 1_000_000, seed=spec["seed"])
    dev = torch.device("cuda", torch.cuda.current_device())
    u = torch.from_numpy(b.u).to(dev)
    v = torch.from_numpy(b.v).to(dev)
    w = torch.from_numpy(b.w).to(dev)
    off = torch.from_numpy(b.edge_offsets).to(dev)
    m = b.m
    ws = torch.empty(pd.workspace_size(m, b.n_trees), dtype=torch.uint8, device=dev)
    ep = torch.empty(m, dtype=torch.int32, device=dev)
    vp = torch.empty(m + b.n_trees, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    tuning = pd.get_tuning()

    def call(kind):
        if kind == "planned":
            pd.dendrogram_batched_planned(u, v, w, off, b.edge_offsets, ws, (ep, vp))
        else:
            pd.dendrogram_batched_async(u, v, w, off, ws, (ep, vp))

    def capture(kind):
        # warm-up on a side stream, then capture the batched call once
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(max(args.warmup, 3)):
                call(kind)
        stream.wait_stream(side)
        torch.cuda.synchronize()
        pd.workspace_status(ws)
        graph = torch.cuda.CUDAGraph()
        pd.profile_start(timing=False)   # counts the kernels the graph holds
        with torch.cuda.graph(graph):
            call(kind)
        kernels = sum(e["kernels"] for e in pd.profile_read().values())
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        pd.workspace_status(ws)
        return graph, kernels

    # the forest-only graph, for comparison (not the headline)
    g_forest, _ = capture("async")
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g_forest.replay()
    ev1.record(stream)
    torch.cuda.synchronize()
    forest_graph_ms = ev0.elapsed_time(ev1) / args.steps
    del g_forest
    g, graph_kernels = capture("planned")
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid).replace("GPU-", "")
    sampler = ClockSampler(gpu_id)
    time.sleep(0.6)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    pd.profile_start(timing=False)
    a = torch.cuda.Event(enable_timing=True)
    z = torch.cuda.Event(enable_timing=True)
    sampler.start()
    a.record(stream)
    for _ in range(args.steps):
        g.replay()
    z.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler.stop()
    pd.workspace_status(ws)
    prof = pd.profile_read()
    ms = a.elapsed_time(z) / args.steps
    if dist:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    if dist:
        tm = torch.tensor([m], device=dev, dtype=torch.float64)
        dist.all_reduce(tm)
        m_all = float(tm.item())
    else:
        m_all = float(m)
    value = m_all / (ms / 1e3)

    # kernel split: blocking batched calls with per-kernel CUDA-event timing
    pd.profile_start(timing=True)
    for _ in range(2):
        _, _, bstats = pd.dendrogram_batched(u, v, w, off, workspace=ws, out=(ep, vp), stats=True)
    torch.cuda.synchronize()
    bprof = pd.profile_read()
    blocking_ms = sum((e["ms"] or 0.0) for e in bprof.values()) / 2
    kern = {k: {"launches": e["launches"] // 2, "ms": e["ms"] / 2}
            for k, e in bprof.items() if e["launches"]}

    # blocking batched calls: small trees one block each, the rest as one forest
    for _ in range(2):
        pd.dendrogram_batched(u, v, w, off, workspace=ws, out=(ep, vp))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        pd.dendrogram_batched(u, v, w, off, workspace=ws, out=(ep, vp))
    torch.cuda.synchronize()
    dispatch_ms = (time.perf_counter() - t0) * 1e3 / args.steps

    # one call per tree: blocking calls, then asynchronous calls back to back
    views = []
    for t in range(b.n_trees):
        e0, e1 = int(b.edge_offsets[t]), int(b.edge_offsets[t + 1])
        views.append((u[e0:e1], v[e0:e1], w[e0:e1], ep[e0:e1], vp[e0 + t:e1 + t + 1]))
    for x in views[:8]:
        pd.dendrogram(x[0], x[1], x[2], workspace=ws, out=(x[3], x[4]))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for x in views:
        pd.dendrogram(x[0], x[1], x[2], workspace=ws, out=(x[3], x[4]))
    torch.cuda.synchronize()
    per_tree_blocking_ms = (time.perf_counter() - t0) * 1e3
    a.record(stream)
    for x in views:
        pd.dendrogram_async(x[0], x[1], x[2], ws, (x[3], x[4]))
    z.record(stream)
    torch.cuda.synchronize()
    per_tree_async_ms = a.elapsed_time(z)
    structure = None
    if args.check:
        # structure of 16 trees (the largest included) from the planned
        # graph's outputs; oracle parity of batches is in the GPU tests
        g.replay()
        torch.cuda.synchronize()
        pd.workspace_status(ws)
        ep_h, vp_h = ep.cpu().numpy(), vp.cpu().numpy()
        rng = np.random.default_rng(spec["seed"] + 99)
        sizes = np.diff(b.edge_offsets)
        pick = sorted(set(rng.choice(b.n_trees, size=min(15, b.n_trees), replace=False).tolist()
                          + [int(np.argmax(sizes))]))
        ok = True
        for t in pick:
            e0, e1 = int(b.edge_offsets[t]), int(b.edge_offsets[t + 1])
            st = dendrogram_structure(b.u[e0:e1], b.v[e0:e1], b.w[e0:e1], ep_h[e0:e1],
                                      vp_h[e0 + t:e1 + t + 1])
            ok = ok and st["ok"]
        structure = {"checks": "root, order, two children, Eq. 1", "trees_checked": len(pick),
                     "ok": bool(ok)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "batched_4096", "n_trees": n_total, "total_edges": int(m_all),
                   "trees_per_gpu": n_trees,
                   "parallelism": ("one GPU" if world == 1 else
                                   f"{world} GPUs, trees sharded largest-first, no collective"),
                   "family": spec["desc"], "seed": spec["seed"],
                   "mode": "pandora_dendrogram_batched_planned captured in a CUDA graph "
                           "(small trees to the single-block solver per size bucket when "
                           "the split pays, the rest as one forest)",
                   "l2": "inputs larger than L2"},
        "per_tree_blocking_ms": per_tree_blocking_ms,
        "per_tree_async_ms": per_tree_async_ms,
        "speedup_vs_per_tree_blocking": per_tree_blocking_ms / ms,
        "speedup_vs_per_tree_async": per_tree_async_ms / ms,
        "gpu_launches": graph_kernels * args.steps,
        "gpu_launches_per_step": graph_kernels,
        "blocking_kernel_ms": blocking_ms,
        "blocking_dispatch_ms": dispatch_ms,
        "forest_async_graph_ms": forest_graph_ms,
        "tuning": tuning,
        "structure": structure,
        "blocking_kernels": kern,
        "levels": bstats["level_edges"],
        "clocks": sampler.summary(),
    }
    if dist and init_dist:
        dist.destroy_process_group()
    return line


def run_serving(args):
    _, rank, _ = dist_setup(args)
    line = measure_serving(args)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_serving(args, n_req=None):
    """Continuous batching under Poisson arrivals (p50/p99 latency, edges/s)
    against one blocking call per request on the same trace."""
    import numpy as np
    import torch
    import paper_2401_06089_gb300 as pd
    from paper_2401_06089_gb300 import inputs
    from paper_2401_06089_gb300.serving import DendrogramServer, Request, run_trace
    world, rank, local = dist_setup(args)
    if world > 1:
        torch.cuda.set_device(local)
    spec = WORKLOADS["serving"]
    rng = np.random.default_rng(spec["seed"])
    n_pool = 40
    sizes = inputs.log_uniform_sizes(rng, n_pool, 1000, 10_000_000)
    pool = []
    for k, n in enumerate(sizes):
        t = inputs.rrt(int(n), seed=int(rng.integers(1 << 30)))
        pool.append((torch.from_numpy(t.u).cuda(), torch.from_numpy(t.v).cuda(),
                     torch.from_numpy(t.w).cuda()))
    torch.cuda.synchronize()
    mean_m = float(np.mean([p[2].numel() for p in pool]))
    budget = 60 << 30

    def trace(n_req, rate, seed):
        r2 = np.random.default_rng(seed)
        pick = r2.integers(0, n_pool, size=n_req)
        arr = (np.cumsum(r2.exponential(1.0 / rate, size=n_req)) if rate else np.zeros(n_req))
        reqs = [Request(i, *pool[int(p)]) for i, p in enumerate(pick)]
        return reqs, arr.tolist()

    def serve(reqs, arr):
        server = DendrogramServer(budget, max_batch_edges=32_000_000, max_batch_trees=1024,
                                  n_streams=3)
        t0 = time.perf_counter()
        res = run_trace(server, reqs, arr)
        wall = time.perf_counter() - t0
        return res, wall, server

    # saturated throughput: a backlog of requests all present at t = 0
    reqs, arr = trace(300, None, 11)
    serve(reqs[:20], arr[:20])   # warm-up
    res, wall, _ = serve(reqs, arr)
    sat = sum(r.m for r in reqs) / wall
    # one blocking call per request on the same backlog
    for r in reqs[:5]:
        pd.dendrogram(r.u, r.v, r.w)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for r in reqs:
        pd.dendrogram(r.u, r.v, r.w)
    torch.cuda.synchronize()
    per_req_wall = time.perf_counter() - t0
    per_req_rate = sum(r.m for r in reqs) / per_req_wall
    # Poisson arrivals at 70% of the saturated rate
    n_req = n_req or args.n or spec["n"]
    rate = 0.7 * sat / mean_m
    reqs, arr = trace(n_req + 200, rate, 12)
    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(0).uuid).replace("GPU-", "")
    sampler = ClockSampler(gpu_id)
    time.sleep(0.6)
    sampler.start()
    pd.profile_start(timing=False)
    res, wall, server = serve(reqs, arr)
    sampler.stop()
    serve_kernels = sum(e["kernels"] for e in pd.profile_read().values())
    res = [r for r in res if r.rid >= 200]
    lat = np.array([r.latency for r in res]) * 1e3
    served_edges = sum(r.edge_parent.numel() for r in res)
    t_first = min(r.t_arrival for r in res)
    t_last = max(r.t_done for r in res)
    line = {
        "metric": METRIC, "value": served_edges / (t_last - t_first), "unit": UNIT,
        "n_gpus": 1, "steps": n_req, "warmup": 200, "ms_per_step": None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": "serving", "requests": n_req, "pool_trees": n_pool,
                   "family": spec["desc"], "mean_edges": mean_m, "arrival_rate_per_s": rate,
                   "hbm_budget_bytes": budget, "streams": 3, "max_batch_edges": 32_000_000},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean())},
        "saturated_edges_per_s": sat,
        "per_request_blocking_edges_per_s": per_req_rate,
        "speedup_saturated_vs_per_request": sat / per_req_rate,
        "max_batches_in_flight": server.max_inflight,
        "gpu_launches": serve_kernels,
        "clocks": sampler.summary(),
    }
    return line


# random 4-/8-byte accesses over vertex-sized arrays (10^8 elements), the
# access pattern of the level kernels; windows of 2^22 elements are the
# pattern of a bucketed pass (a bucket that stays in L2)
MEMBENCH_CASES = [
    ("gather32", 10**8, 0), ("gather64", 10**8, 0), ("scatter32", 10**8, 0),
    ("scatter64", 10**8, 0), ("atomicmin64", 10**8, 0), ("gather64", 10**8, 1 << 22),
    ("atomicmin64", 10**8, 1 << 22), ("gather32", 10**7, 0), ("copy32", 10**8, 0),
]


def measure_random_access(torch, pd, n_access=1 << 27, reps=5, blocks_per_sm=8,
                          cases=MEMBENCH_CASES):
    """Accesses per second of each random-access kind (CUDA events on the
    launching stream, mean of `reps` launches after one warm-up)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    out = []
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    for kind, n, window in cases:
        width = 8 if kind.endswith("64") else 4
        buf = torch.zeros(n, dtype=torch.int64 if width == 8 else torch.int32, device=dev)
        if kind == "atomicmin64":
            buf.fill_(-1)   # all ones: every atomic has something to lower at first
        dst = torch.empty(n, dtype=torch.int32, device=dev) if kind == "copy32" else None
        acc = n if kind == "copy32" else n_access
        pd.membench(kind, buf, n_access=acc, window=window, dst=dst, sink=sink,
                    blocks_per_sm=blocks_per_sm)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for r in range(reps):
            pd.membench(kind, buf, n_access=acc, window=window, seed=r + 1, dst=dst, sink=sink,
                        blocks_per_sm=blocks_per_sm)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / reps
        moved = acc * (2 * width if kind == "copy32" else width)
        out.append({"kind": kind, "elem_bytes": width, "array_bytes": n * width,
                    "window_bytes": (window or n) * width, "accesses": acc, "ms": ms,
                    "g_access_per_s": acc / ms / 1e6, "useful_gbs": moved / ms / 1e6})
        del buf, dst
    return out


def run_membench(args):
    import torch
    import paper_2401_06089_gb300 as pd
    pd.load_library()
    res = {}
    for bps in args.membench_bps:
        res[f"bps{bps}"] = measure_random_access(torch, pd, reps=args.membench_reps,
                                                 blocks_per_sm=bps)
    peak, kind = load_peaks()
    print(json.dumps({"metric": "random-access ceiling (pandora_membench)",
                      "unit": "G accesses/s", "hbm_peak_gbs": peak, "peak_source": kind,
                      "results": res}), flush=True)


# What bounds the spanning-tree traversals (k-NN and Boruvka queries, over
# 90% of the call; ncu summary in profiles/emst_gmm_4e6.md): neither DRAM nor
# arithmetic, so no roofline fraction applies.
EMST_BOUND = {"kind": "latency",
              "detail": "divergent BVH traversals: k-NN kernel at 1e6 points 0.2% of DRAM peak, "
                        "L1 hit rate 94%, 9.9 of 32 lanes active per instruction",
              "profile": "profiles/emst_gmm_4e6.md"}


def run_emst(args):
    import numpy as np
    import torch
    import paper_2401_06089_gb300 as pd
    from paper_2401_06089_gb300 import inputs
    pts = torch.from_numpy(inputs.gmm_points(args.emst, 3).astype(np.float32)).cuda()
    for _ in range(max(args.warmup, 1)):
        pd.mr_emst(pts, 16)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        pd.mr_emst(pts, 16)
        torch.cuda.synchronize()
        times.append((time.perf_counter() - t0) * 1e3)
    ms = statistics.median(times)
    print(json.dumps({"metric": "mutual-reachability MST points/s (pandora_mr_emst)",
                      "value": args.emst / (ms / 1e3), "unit": "points/s", "ms": ms,
                      "steps": args.steps, "n_points": args.emst, "min_pts": 16,
                      "data": "synthetic 32-component Gaussian mixture, seed 3",
                      "timing": "wall clock around the blocking call, median",
                      "bound": EMST_BOUND}), flush=True)


def main():
    args = parse_args()
    if args.membench:
        return run_membench(args)
    if args.emst:
        return run_emst(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload.startswith("batched"):
        return run_batched(args)
    import numpy as np
    import torch
    import paper_2401_06089_gb300 as pd
    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    dev = torch.device("cuda", torch.cuda.current_device())
    spec = WORKLOADS[args.workload]
    t = make_tree(spec, args.n)
    m = t.m
    pd.load_library()

    u = torch.from_numpy(t.u).to(dev)
    v = torch.from_numpy(t.v).to(dev)
    w = torch.from_numpy(t.w).to(dev)
    ws = torch.empty(pd.workspace_size(m), dtype=torch.uint8, device=dev)
    ep = torch.empty(m, dtype=torch.int32, device=dev)
    vp = torch.empty(m + 1, dtype=torch.int32, device=dev)

    _, _, stats = pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp), stats=True)
    for _ in range(max(args.warmup, 3)):
        pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
    torch.cuda.synchronize()

    gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid).replace("GPU-", "")
    sampler = ClockSampler(gpu_id)
    time.sleep(0.6)   # let nvidia-smi start sampling
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    pd.profile_start(timing=True)
    stream = torch.cuda.current_stream(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler.start()
    for k in range(args.steps):
        evs[k][0].record(stream)
        if args.async_api:
            pd.dendrogram_async(u, v, w, ws, (ep, vp))
        else:
            pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    sampler.stop()
    prof = pd.profile_read()
    timing_note = "CUDA events inside the timed region"
    graph_ms = None
    if args.async_api:
        # the asynchronous path only counts launches; time the kernels on
        # blocking calls of the same tree right after the timed region
        launches_async = sum(e["kernels"] for e in prof.values())
        pd.profile_start(timing=True)
        for _ in range(args.steps):
            pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
        torch.cuda.synchronize()
        prof = pd.profile_read()
        for e in prof.values():
            e["launches_async"] = None
        timing_note = ("kernel split from blocking calls after the timed region; "
                       f"{launches_async} kernel launches in the timed region")
        # the same call captured once in a CUDA graph and replayed
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            pd.dendrogram_async(u, v, w, ws, (ep, vp))
        stream.wait_stream(side)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            pd.dendrogram_async(u, v, w, ws, (ep, vp))
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        ga = torch.cuda.Event(enable_timing=True)
        gb = torch.cuda.Event(enable_timing=True)
        ga.record(stream)
        for _ in range(args.steps):
            g.replay()
        gb.record(stream)
        torch.cuda.synchronize()
        graph_ms = ga.elapsed_time(gb) / args.steps
        pd.workspace_status(ws)
        del g
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    if dist:
        tt = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    if dist:
        tm = torch.tensor([m], device=dev, dtype=torch.float64)
        dist.all_reduce(tm)
        m_all = float(tm.item())
    else:
        m_all = float(m)
    value = m_all / (ms / 1e3)

    # ---- roofline of the dominant kernel --------------------------------
    peak, peak_kind = load_peaks()
    n_passes_w = prof["onesweep_weights"]["launches"] // max(args.steps, 1)
    l0 = args.steps if m + 1 >= FLAGGED_LEVEL0_MIN_VERTICES else 0
    m1 = stats["level_edges"][1] if len(stats["level_edges"]) > 1 else 0
    kernels = {}
    for name, e in prof.items():
        if e["launches"] == 0:
            continue
        b = model_bytes(name, e, m, n_passes_w, l0, m1) if name != "onesweep_weights" else \
            sort_weight_bytes(m, n_passes_w) * args.steps
        kernels[name] = {"launches": e["launches"], "ms": e["ms"],
                         "share": e["ms"] / (ms * args.steps) if e["ms"] else None,
                         "gbs": b / (e["ms"] / 1e3) / 1e9 if e["ms"] else None}
    dom = max(kernels, key=lambda k: kernels[k]["ms"] or 0.0)
    dom_e = prof[dom]
    dom_bytes_total = (sort_weight_bytes(m, n_passes_w) * args.steps if dom == "onesweep_weights"
                       else model_bytes(dom, dom_e, m, n_passes_w, l0, m1))
    per_launch_bytes = dom_bytes_total / dom_e["launches"]
    per_launch_ms = dom_e["ms"] / dom_e["launches"]
    achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
    traffic = recorded_traffic(dom)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "kernel": dom,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": per_launch_bytes}
    path_bytes = sum((sort_weight_bytes(m, n_passes_w) * args.steps if k == "onesweep_weights"
                      else model_bytes(k, prof[k], m, n_passes_w, l0, m1)) for k in kernels)
    path_roofline = path_bytes / args.steps / (ms / 1e3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": config_of(args, spec),
        "roofline": roofline,
        "path_model_gbs": path_roofline,
        "path_model_frac": path_roofline / peak,
        "gpu_launches": sum(e["kernels"] for e in prof.values()),
        "gpu_launches_per_step": sum(e["kernels"] for e in prof.values()) / args.steps,
        "kernels": kernels,
        "kernel_timing": timing_note,
        "api": "pandora_dendrogram_async" if args.async_api else "pandora_dendrogram",
        "graph_ms_per_step": graph_ms if args.async_api else None,
        "levels": stats["level_edges"],
        "skewness": skewness(ep, vp),
        "clocks": sampler.summary(),
    }

    # ---- end to end through the public API with host buffers -------------
    if not args.no_e2e:
        uh = torch.from_numpy(t.u).pin_memory()
        vh = torch.from_numpy(t.v).pin_memory()
        wh = torch.from_numpy(t.w).pin_memory()
        eph = torch.empty(m, dtype=torch.int32).pin_memory()
        vph = torch.empty(m + 1, dtype=torch.int32).pin_memory()
        k_e2e = max(3, min(args.steps, 10))
        t_list = []
        # the device-resident call's outputs, to check the host path against
        pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
        ep_ref, vp_ref = ep.cpu(), vp.cpu()
        torch.cuda.synchronize()
        for k in range(k_e2e + 3):   # three untimed warm-up calls
            t0 = time.perf_counter()
            pd.dendrogram_host(uh, vh, wh, out=(eph, vph))
            if k >= 3:
                t_list.append((time.perf_counter() - t0) * 1e3)
        e2e_ms = sum(t_list) / len(t_list)
        e2e_same = bool(torch.equal(eph, ep_ref) and torch.equal(vph, vp_ref))
        # this process's host link, measured on the same pinned buffers: the
        # end-to-end time moves with it from box to box
        link = {}
        for name, dst, src in (("h2d_gbs", ep, eph), ("d2h_gbs", eph, ep)):
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            link[name] = round(3 * 4 * m / (time.perf_counter() - t0) / 1e9, 1)
        if dist:
            tt = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_ms = float(tt.item())
        line["e2e"] = {"value": world * m / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                       "h2d_bytes_per_step": 12 * m, "d2h_bytes_per_step": 4 * m + 4 * (m + 1),
                       "api": "pandora_dendrogram_host (pinned host buffers in and out, "
                              "wall clock around the blocking call)",
                       "outputs_equal_device_call": e2e_same, "host_link": link}

    # ---- the path family at the same size --------------------------------
    if not args.no_extra and args.workload == "rrt_1e8":
        spec2 = WORKLOADS["path_1e8"]
        t2 = make_tree(spec2, args.n)
        u2 = torch.from_numpy(t2.u).to(dev)
        v2 = torch.from_numpy(t2.v).to(dev)
        w2 = torch.from_numpy(t2.w).to(dev)
        for _ in range(args.warmup):
            pd.dendrogram(u2, v2, w2, workspace=ws, out=(ep, vp))
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        k2 = max(3, args.steps // 2)
        a.record(stream)
        for _ in range(k2):
            pd.dendrogram(u2, v2, w2, workspace=ws, out=(ep, vp))
        b.record(stream)
        b.synchronize()
        ms2 = a.elapsed_time(b) / k2
        _, _, st2 = pd.dendrogram(u2, v2, w2, workspace=ws, out=(ep, vp), stats=True)
        line["path_skewed_1e8"] = {"value": t2.m / (ms2 / 1e3), "unit": UNIT, "ms_per_step": ms2,
                                   "steps": k2, "levels": st2["level_edges"],
                                   "skewness": skewness(ep, vp)}
        del u2, v2, w2

    # ---- CPU oracle on a bounded sample (rank 0, N = 1) -------------------
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baseline(spec, args.n)
    # ---- HDBSCAN* flat clusters on the same dendrogram (optional) ----------
    if args.flat and rank == 0:
        pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        labels = pd.hdbscan_labels(ep, vp, w, args.flat)
        torch.cuda.synchronize()
        # the library's pool keeps what the call took: the drop in free memory
        # is the call's scratch high-water mark (outputs come from torch)
        flat_scratch = free0 - torch.cuda.mem_get_info()[0] - labels.numel() * 4
        for _ in range(max(args.warmup, 3)):
            labels = pd.hdbscan_labels(ep, vp, w, args.flat)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        k3 = max(3, args.steps // 2)
        a.record(stream)
        for _ in range(k3):
            labels = pd.hdbscan_labels(ep, vp, w, args.flat)
        b.record(stream)
        b.synchronize()
        ms3 = a.elapsed_time(b) / k3
        lab_np = labels.cpu().numpy()
        line["flat_clusters"] = {"min_cluster_size": args.flat, "ms_per_call": ms3,
                                 "scratch_bytes": int(flat_scratch),
                                 "points_per_s": (m + 1) / (ms3 / 1e3), "steps": k3,
                                 "clusters": int(lab_np.max()) + 1,
                                 "noise_fraction": float((lab_np < 0).mean())}
    if args.check and rank == 0:
        gep, gvp = pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
        line["structure"] = dendrogram_structure(t.u, t.v, t.w, gep.cpu().numpy(),
                                                 gvp.cpu().numpy())
    # ---- measured random-access ceilings (the level kernels' bound) -------
    if not args.no_extra and rank == 0:
        ra = measure_random_access(torch, pd, reps=3, blocks_per_sm=8)
        line["random_access_ceiling"] = {
            "unit": "G accesses/s", "kernel": "pandora_membench (one launch per pattern, "
                                              "2^27 accesses at hashed positions)",
            "patterns": {f"{r['kind']} over {r['array_bytes'] // 10**6} MB" +
                         (f", {r['window_bytes'] // 2**20} MiB windows"
                          if r["window_bytes"] < r["array_bytes"] else ""):
                         round(r["g_access_per_s"], 2) for r in ra if r["kind"] != "copy32"}}

    # ---- the other configurations, each as a sub-record -----------------
    if not args.no_extra and args.workload == "rrt_1e8" and args.n is None:
        line["rrt_1e4"] = measure_rrt_1e4(pd, torch, args)
        line["batched_4096"] = summarize_batched(measure_batched(args, init_dist=False))
        torch.cuda.empty_cache()
        line["serving"] = summarize_serving(measure_serving(args))
        torch.cuda.empty_cache()
        line["hdbscan"] = measure_hdbscan(pd, torch, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
