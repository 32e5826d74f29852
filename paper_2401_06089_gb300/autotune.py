"""Autotuner for the small-tree settings (block size per size bucket, the
single-block solver's cutoff, the batch-split threshold).

    python -m paper_2401_06089_gb300.autotune --out paper_2401_06089_gb300/tuning_gb300.json

For every size bucket k (trees of 2^k .. 2^(k+1)-1 edges) it times batches of
such trees through ``pandora_dendrogram_batched_planned``:

* with the single-block solver at 256, 512 and 1024 threads per block (the
  whole batch then runs in the solver, one block per tree), and
* with the solver off (the same batch as one forest through the pipeline).

The fastest block size is kept per bucket; the cutoff is the top of the last
bucket (from bucket 0 up) in which the solver beats the pipeline.  The split
threshold compares what splitting a mixed batch costs per large-tree edge
(packing the large trees into one forest and copying their results back)
with what it saves per small-tree edge (pipeline time minus solver time):
a batch is split when its small trees hold at least the break-even share of
its edges.

Every timing is CUDA events on the launching stream after warm-up calls; the
results and the raw timings go to the JSON file, which ``load_tuning`` (and
``load_library``, for the file shipped beside the package) applies.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import _binding as B
from . import inputs

THREADS = (256, 512, 1024)
CAP = B.SMALL_CAP


def _bucket_sizes(k: int, rng, target_edges: int):
    lo, hi = (1 << k), min((1 << (k + 1)) - 1, CAP)
    if k == 0:
        lo, hi = 1, 1
    n_trees = int(min(50_000, max(1024, target_edges // max(lo, 1))))
    edges = rng.integers(lo, hi + 1, size=n_trees)
    return edges + 1   # vertex counts


class _Runner:
    """Device copies of one batch and a timer for the planned call."""

    def __init__(self, b):
        import torch
        self.torch = torch
        self.b = b
        dev = torch.device("cuda")
        self.u = torch.from_numpy(b.u).to(dev)
        self.v = torch.from_numpy(b.v).to(dev)
        self.w = torch.from_numpy(b.w).to(dev)
        self.off = torch.from_numpy(b.edge_offsets).to(dev)
        self.ws = torch.empty(B.workspace_size(b.m, b.n_trees), dtype=torch.uint8, device=dev)
        self.ep = torch.empty(b.m, dtype=torch.int32, device=dev)
        self.vp = torch.empty(b.m + b.n_trees, dtype=torch.int32, device=dev)

    def call(self):
        B.dendrogram_batched_planned(self.u, self.v, self.w, self.off, self.b.edge_offsets,
                                     self.ws, (self.ep, self.vp))

    def time_ms(self, reps: int = 5, warm: int = 2) -> float:
        torch = self.torch
        for _ in range(warm):
            self.call()
        torch.cuda.synchronize()
        st = B.workspace_status(self.ws, raise_on_error=False)
        if st:
            raise B.PandoraError(st, "autotune batch")
        a = torch.cuda.Event(enable_timing=True)
        z = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            self.call()
        z.record()
        torch.cuda.synchronize()
        return a.elapsed_time(z) / reps

    def outputs(self):
        return self.ep.cpu().numpy(), self.vp.cpu().numpy()


def choose_threads_and_cutoff(buckets):
    """Fastest block size per bucket; the cutoff is the top of the last bucket,
    counting up from bucket 0, in which the solver beats the pipeline."""
    threads = [row["best_threads"] for row in buckets]
    cutoff = 0
    for row in buckets:
        if row["solver_ms"][str(row["best_threads"])] < row["pipeline_ms"]:
            cutoff = min(CAP, (1 << (row["bucket"] + 1)) - 1)
        else:
            break
    return threads, cutoff


def choose_split_permille(buckets, cutoff, pack_ns_per_large_edge):
    """Split a mixed batch when its small trees hold at least the share s of
    its edges at which the saving equals the packing cost:
    s * saving = (1 - s) * pack, with saving the median (pipeline - solver)
    time per edge over the buckets under the cutoff.  Returns (saving, per
    mille); no saving means never split a mixed batch (1000)."""
    small_rows = [row for row in buckets if row["bucket"] >= 1 and
                  (1 << row["bucket"]) <= max(cutoff, 1)]
    if small_rows:
        saving = float(np.median([row["pipeline_ns_per_edge"] - row["solver_ns_per_edge"]
                                  for row in small_rows]))
    else:
        saving = 0.0
    if saving <= 0:
        return saving, 1000
    g = pack_ns_per_large_edge
    return saving, int(min(max(math.ceil(1000 * g / (g + saving) - 1e-9), 0), 1000))


def tune(target_edges: int = 2_000_000, seed: int = 7, verbose: bool = True) -> dict:
    import torch
    B.load_library()
    saved = B.get_tuning()
    rng = np.random.default_rng(seed)
    buckets = []
    try:
        for k in range(13):
            sizes = _bucket_sizes(k, rng, target_edges)
            b = inputs.batch(len(sizes), 1, 1, seed=seed + k, sizes=sizes)
            r = _Runner(b)
            per = {}
            ref = None
            for t in THREADS:
                B.set_tuning(CAP, [t] * 13, 0)
                per[t] = r.time_ms()
                out = r.outputs()
                if ref is None:
                    ref = out
                elif not (np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])):
                    raise RuntimeError(f"bucket {k}: block sizes disagree")
            B.set_tuning(0, None, 0)
            forest = r.time_ms()
            out = r.outputs()
            if not (np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])):
                raise RuntimeError(f"bucket {k}: solver and pipeline disagree")
            best = min(per, key=per.get)
            row = {"bucket": k, "trees": int(b.n_trees), "edges": int(b.m),
                   "solver_ms": {str(t): per[t] for t in THREADS}, "pipeline_ms": forest,
                   "best_threads": best,
                   "solver_ns_per_edge": 1e6 * per[best] / max(b.m, 1),
                   "pipeline_ns_per_edge": 1e6 * forest / max(b.m, 1)}
            buckets.append(row)
            if verbose:
                print(json.dumps(row), flush=True)
            del r
            torch.cuda.empty_cache()

        threads, cutoff = choose_threads_and_cutoff(buckets)

        # split threshold: packing cost per large-tree edge against the saving
        # per small-tree edge, on a batch of a few large trees and many small ones
        big = np.full(8, 500_001, np.int64)
        small = rng.integers(max(cutoff // 4, 2), max(cutoff, 2) + 1, size=2000) + 1
        sizes = np.concatenate([big, small])
        rng.shuffle(sizes)
        b = inputs.batch(len(sizes), 1, 1, seed=seed + 100, sizes=sizes)
        B.set_tuning(cutoff, threads, 0)
        B.profile_start(timing=True)
        import torch as _t
        u, v, w, off = (_t.from_numpy(x).cuda() for x in (b.u, b.v, b.w, b.edge_offsets))
        for _ in range(3):
            B.dendrogram_batched(u, v, w, off)
        _t.cuda.synchronize()
        prof = B.profile_read()
        large_edges = int(8 * 500_000)
        pack_ms = (prof.get("gather_scatter", {}).get("ms") or 0.0) / 3
        g = 1e6 * pack_ms / large_edges                   # ns per large-tree edge
        saving, permille = choose_split_permille(buckets, cutoff, g)
        result = {
            "small_max_edges": int(cutoff),
            "small_threads": [int(t) for t in threads],
            "split_min_permille": int(min(max(permille, 0), 1000)),
            "measured": {
                "device": _t.cuda.get_device_name(0),
                "date": time.strftime("%Y-%m-%d %H:%M:%S"),
                "target_edges_per_bucket": target_edges,
                "pack_ns_per_large_edge": g,
                "saving_ns_per_small_edge": saving,
                "buckets": buckets,
            },
        }
        return result
    finally:
        B.set_tuning(saved["small_max_edges"], saved["small_threads"], saved["split_min_permille"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "tuning_gb300.json"))
    ap.add_argument("--target-edges", type=int, default=2_000_000)
    args = ap.parse_args()
    res = tune(args.target_edges)
    with open(args.out, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps({k: res[k] for k in ("small_max_edges", "small_threads",
                                          "split_min_permille")}))


if __name__ == "__main__":
    main()
