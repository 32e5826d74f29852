"""Sharding a batch of trees across GPUs (one process per GPU).

Trees are independent problems: a tree's dendrogram depends on that tree
only, so a batch splits by whole trees with no exchange between ranks.  Each
rank runs the batched entry point on its own sub-batch; an optional final
gather of the outputs is host-side.  A single tree does not shard (a parent
can come from anywhere in the tree and the method sorts all its edges
globally), so single-tree work runs as independent replicas.

The split is greedy longest-processing-time: trees in decreasing edge count,
each to the rank with the fewest edges so far; the cost of a tree is close to
linear in its edges.  Each rank keeps its trees in batch order.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence

import numpy as np


def shard_trees(edge_counts: Sequence[int], world: int) -> List[np.ndarray]:
    """Tree indices of every rank (sorted), balancing edge counts."""
    if world < 1:
        raise ValueError("world must be >= 1")
    m = np.asarray(edge_counts, dtype=np.int64)
    order = np.argsort(-m, kind="stable")
    heap = [(0, r) for r in range(world)]
    owned: List[list] = [[] for _ in range(world)]
    for t in order:
        load, r = heapq.heappop(heap)
        owned[r].append(int(t))
        heapq.heappush(heap, (load + int(m[t]), r))
    return [np.array(sorted(o), dtype=np.int64) for o in owned]


def sub_batch(u, v, w, edge_offsets, trees: np.ndarray):
    """Host arrays (u, v, w, offsets) of the trees `trees` of a batch, packed
    in that order; ids stay tree-local."""
    off = np.asarray(edge_offsets, dtype=np.int64)
    sizes = off[trees + 1] - off[trees]
    new_off = np.zeros(len(trees) + 1, dtype=np.int64)
    np.cumsum(sizes, out=new_off[1:])
    if len(trees):
        idx = np.concatenate([np.arange(off[t], off[t + 1]) for t in trees])
    else:
        idx = np.zeros(0, dtype=np.int64)
    return (np.asarray(u)[idx], np.asarray(v)[idx], np.asarray(w)[idx], new_off)


def merge_outputs(edge_offsets, shards: Sequence[np.ndarray], outputs):
    """Reassemble the batch outputs from the ranks' sub-batch outputs
    (`outputs[r] = (edge_parent, vertex_parent)` of rank r's sub-batch)."""
    off = np.asarray(edge_offsets, dtype=np.int64)
    n_trees = len(off) - 1
    m = int(off[-1])
    ep = np.empty(m, dtype=np.int32)
    vp = np.empty(m + n_trees, dtype=np.int32)
    seen = np.zeros(n_trees, dtype=bool)
    for trees, (sep, svp) in zip(shards, outputs):
        k0 = 0
        for j, t in enumerate(trees):
            mt = int(off[t + 1] - off[t])
            ep[off[t]:off[t + 1]] = sep[k0:k0 + mt]
            vp[off[t] + t:off[t + 1] + t + 1] = svp[k0 + j:k0 + j + mt + 1]
            k0 += mt
            seen[t] = True
    if not seen.all():
        raise ValueError("some trees belong to no shard")
    return ep, vp
