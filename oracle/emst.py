"""Mutual-reachability minimum spanning tree of a point set (CPU oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain numpy, O(n^2),
no shared code with the GPU library.

The step before the dendrogram in the paper's HDBSCAN* pipeline (Section 6.5):
the minimum spanning tree of the complete graph on the points whose edge
weights are mutual-reachability distances.  Written out (reading R12 for
minPts):

* d(a, b) = Euclidean distance, in float64 (sqrt of the sum of squared
  coordinate differences, coordinates taken exactly from their input type);
* core(a) = d(a, the min_pts-th nearest point to a, counting a itself), so
  min_pts = 1 gives 0;
* mr(a, b) = max(core(a), core(b), d(a, b));
* the tree: Prim's algorithm from point 0 over the complete graph with
  weights mr; among equally light candidates the one reached first wins
  (smaller vertex id, then the earlier tree vertex).  A minimum spanning tree
  is unique only up to ties, but the sorted list of its weights is not: it is
  what a different construction must reproduce.
"""
from __future__ import annotations

import numpy as np


def pair_distance(points, a: int, b: int) -> float:
    diff = points[a] - points[b]
    return float(np.sqrt(np.dot(diff, diff)))


def core_distances(points, min_pts: int) -> np.ndarray:
    """core(a) for every point, float64."""
    p = np.asarray(points, np.float64)
    n = len(p)
    if not 1 <= min_pts <= n:
        raise ValueError("min_pts must be in [1, number of points]")
    core = np.zeros(n)
    for a in range(n):
        diff = p - p[a]
        d = np.sqrt(np.einsum("ij,ij->i", diff, diff))
        core[a] = np.sort(d)[min_pts - 1]          # d[a] = 0 is counted
    return core


def mr_emst(points, min_pts: int):
    """(u, v, w): the n - 1 tree edges in the order Prim adds them (u already
    in the tree, v the vertex added), w their float64 mutual-reachability
    weights."""
    p = np.asarray(points, np.float64)
    n = len(p)
    if n == 0:
        raise ValueError("no points")
    core = core_distances(p, min_pts)
    in_tree = np.zeros(n, bool)
    best = np.full(n, np.inf)
    link = np.full(n, -1, np.int64)
    best[0] = 0.0
    us, vs, ws = [], [], []
    for _ in range(n):
        cand = np.where(in_tree, np.inf, best)
        x = int(np.argmin(cand))                   # first index among equals
        in_tree[x] = True
        if link[x] >= 0:
            us.append(int(link[x]))
            vs.append(x)
            ws.append(float(best[x]))
        diff = p - p[x]
        d = np.sqrt(np.einsum("ij,ij->i", diff, diff))
        mr = np.maximum(np.maximum(core, core[x]), d)
        upd = (~in_tree) & (mr < best)             # strict: an earlier link stays
        best[upd] = mr[upd]
        link[upd] = x
    return (np.array(us, np.int64), np.array(vs, np.int64), np.array(ws, np.float64))


def mr_matrix(points, min_pts: int) -> np.ndarray:
    """The complete mutual-reachability weight matrix (diagonal 0), float64."""
    p = np.asarray(points, np.float64)
    core = core_distances(p, min_pts)
    diff = p[:, None, :] - p[None, :, :]
    d = np.sqrt(np.einsum("ijk,ijk->ij", diff, diff))
    m = np.maximum(np.maximum(core[:, None], core[None, :]), d)
    np.fill_diagonal(m, 0.0)
    return m


# ---------------------------------------------------------------------------
# Float32 reading of the same tree (the arithmetic a float32 construction on
# the GPU performs), written out step by step:
#
# * d2(a, b) = ((dx*dx + dy*dy) + dz*dz) with dx = a.x - b.x etc., every
#   operation a float32 operation rounded to nearest (no fused multiply-add),
#   in that order; in other dimensions the squares are added left to right;
# * core2(a) = the min_pts-th smallest of d2(a, p) over all points p,
#   counting d2(a, a) = 0;
# * mr2(a, b) = max(core2(a), core2(b), d2(a, b)) (a maximum of float32
#   values, so exact), and the weight of the edge is the float32 square root
#   of mr2 (correctly rounded);
# * edges are totally ordered by (mr2, smaller endpoint, larger endpoint); the
#   minimum spanning tree under a strict total order is unique, and Prim's
#   algorithm below adds, at every step, the least edge leaving the tree in
#   that order.
# ---------------------------------------------------------------------------
def sq_distances_f32(points, a: int) -> np.ndarray:
    """d2(a, p) for every p, float32, in the operation order above."""
    p = np.asarray(points, np.float32)
    acc = None
    for k in range(p.shape[1]):
        dk = p[:, k] - p[a, k]                     # float32 subtraction
        sq = dk * dk                               # float32 product
        acc = sq if acc is None else acc + sq      # float32 sum, left to right
    return acc


def core_sq_distances_f32(points, min_pts: int) -> np.ndarray:
    """core2(a) for every point, float32."""
    p = np.asarray(points, np.float32)
    n = len(p)
    if not 1 <= min_pts <= n:
        raise ValueError("min_pts must be in [1, number of points]")
    core2 = np.zeros(n, np.float32)
    for a in range(n):
        d2 = sq_distances_f32(p, a)
        core2[a] = np.partition(d2, min_pts - 1)[min_pts - 1]
    return core2


def mr_emst_f32(points, min_pts: int):
    """(u, v, mr2): the n - 1 tree edges of the float32 reading, in the order
    Prim adds them (u in the tree, v the vertex added), mr2 float32; the
    weight of an edge is np.sqrt(mr2) in float32."""
    p = np.asarray(points, np.float32)
    n = len(p)
    if n == 0:
        raise ValueError("no points")
    core2 = core_sq_distances_f32(p, min_pts)
    in_tree = np.zeros(n, bool)
    # least known edge from each vertex to the tree: (weight, lo, hi)
    bw = np.full(n, np.inf, np.float32)
    blo = np.full(n, n, np.int64)
    bhi = np.full(n, n, np.int64)
    link = np.full(n, -1, np.int64)
    ids = np.arange(n, dtype=np.int64)
    us, vs, ws = [], [], []
    x = 0
    for step in range(n):
        in_tree[x] = True
        if step > 0:
            us.append(int(link[x]))
            vs.append(x)
            ws.append(bw[x])
        d2 = sq_distances_f32(p, x)
        w2 = np.maximum(np.maximum(core2, core2[x]), d2)
        lo = np.minimum(ids, x)
        hi = np.maximum(ids, x)
        better = (w2 < bw) | ((w2 == bw) & ((lo < blo) | ((lo == blo) & (hi < bhi))))
        better &= ~in_tree
        bw[better] = w2[better]
        blo[better] = lo[better]
        bhi[better] = hi[better]
        link[better] = x
        if step + 1 < n:
            out = np.flatnonzero(~in_tree)
            # the least (weight, lo, hi) among the vertices outside the tree
            order = np.lexsort((bhi[out], blo[out], bw[out]))
            x = int(out[order[0]])
    return (np.array(us, np.int64), np.array(vs, np.int64), np.array(ws, np.float32))
