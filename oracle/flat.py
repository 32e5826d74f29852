"""HDBSCAN* flat clusters from a single-linkage dendrogram (CPU oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring): plain Python loops over
the dendrogram, no shared code with the GPU library.

The paper's HDBSCAN* pipeline (Section 6.5) ends with the optional step that
turns the hierarchy into non-overlapping flat clusters and marks the rest as
noise, as defined by Campello et al. (2015): clusters are the parts of the
tree that stay at least ``min_cluster_size`` points large as edges are removed
from the heaviest down, each cluster is scored by its stability, and the
non-overlapping set of clusters of largest total stability is kept ("excess of
mass").  Written out:

* lambda(e) = 1 / w(e) in float64 (weights must be positive and finite);
* the tree is walked from the root edge; the root starts cluster 0, born at
  lambda 0.  At an edge e of cluster C with children c1, c2 (edges or
  vertices, sizes s1, s2 in leaves):
  - s1 >= mcs and s2 >= mcs: C ends, each child starts a new cluster (child
    of C) born at lambda(e);
  - exactly one child large: it continues C; the other child's leaves leave C
    at lambda(e);
  - neither large: every leaf under e leaves C at lambda(e);
* stability(C) is the sum, over C's points, of how long each point stays in
  C: for a leaf x that leaves C, the float64 term
  fl(lambda_leave(x) - lambda_birth(C)); for the points of a child cluster D,
  size(D) copies of fl(lambda_birth(D) - lambda_birth(C)).  The sum is taken
  exactly (rational arithmetic) and rounded once to the nearest float64, so it
  does not depend on any summation order;
* selection, children before parents, over every cluster but the root (the
  whole data set is not a candidate): a cluster with no child cluster is
  selected and scores its stability; otherwise its children's scores are
  summed exactly (no rounding: a score is an exact sum of float64
  stabilities, so the selection is the exact optimum of the total
  stability) and the cluster is selected, and its descendants deselected,
  when its stability is at least that sum (so a parent wins a tie), scoring
  its stability, else it scores the sum;
* label of a vertex: the selected cluster among the cluster it leaves and that
  cluster's ancestors, or -1 (noise); selected clusters are numbered 0, 1, ...
  in increasing order of their smallest vertex id.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _round(total: Fraction) -> float:
    # int / int true division in Python is correctly rounded
    return total.numerator / total.denominator


def hdbscan_labels(edge_parent, vertex_parent, w, min_cluster_size, members: bool = False):
    """Returns (labels int32[n], info) for a dendrogram of m edges and
    n = m + 1 vertices.  info["clusters"]: per cluster (in creation order,
    cluster 0 the root) its starting node ("e", edge) or the root edge, parent
    cluster, birth lambda, size, stability, score (exact, a Fraction),
    selection and label (-1 unless selected); with
    ``members`` also its sorted vertex ids."""
    ep = np.asarray(edge_parent, dtype=np.int64)
    vp = np.asarray(vertex_parent, dtype=np.int64)
    w = np.asarray(w, dtype=np.float32)
    m = len(ep)
    n = m + 1
    mcs = int(min_cluster_size)
    if mcs < 2:
        raise ValueError("min_cluster_size must be at least 2")
    if m == 0:
        return np.full(1, -1, np.int32), {"clusters": []}
    wd = w.astype(np.float64)
    if not np.all(np.isfinite(wd)) or np.any(wd <= 0):
        raise ValueError("weights must be positive and finite")
    lam = [1.0 / float(x) for x in wd]
    # children of every edge: ("e", f) for edges, ("v", x) for vertices
    children = [[] for _ in range(m)]
    root = -1
    for f in range(m):
        if ep[f] < 0:
            root = f
        else:
            children[int(ep[f])].append(("e", f))
    for x in range(n):
        children[int(vp[x])].append(("v", x))
    assert all(len(c) == 2 for c in children), "not a binary dendrogram"
    # leaf counts, children before parents (iterative post-order)
    size = np.zeros(m, np.int64)
    order = []
    stack = [root]
    while stack:
        e = stack.pop()
        order.append(e)
        for kind, c in children[e]:
            if kind == "e":
                stack.append(c)
    for e in reversed(order):
        size[e] = sum(1 if kind == "v" else size[c] for kind, c in children[e])

    def csize(kind, c):
        return 1 if kind == "v" else int(size[c])

    def leaves(kind, c):
        if kind == "v":
            return [c]
        out = []
        st = [c]
        while st:
            f = st.pop()
            for k2, c2 in children[f]:
                if k2 == "v":
                    out.append(c2)
                else:
                    st.append(c2)
        return out

    clusters = [{"edge": root, "parent": -1, "birth": 0.0, "size": int(size[root]),
                 "children": [], "leaving": []}]
    # top-down walk: (edge, cluster)
    stack = [(root, 0)]
    while stack:
        e, ci = stack.pop()
        (k1, c1), (k2, c2) = children[e]
        big1 = csize(k1, c1) >= mcs
        big2 = csize(k2, c2) >= mcs
        if big1 and big2:
            for kind, c in ((k1, c1), (k2, c2)):
                clusters.append({"edge": c, "parent": ci, "birth": lam[e],
                                 "size": csize(kind, c), "children": [], "leaving": []})
                di = len(clusters) - 1
                clusters[ci]["children"].append(di)
                stack.append((c, di))
            continue
        for kind, c, big in ((k1, c1, big1), (k2, c2, big2)):
            if big:
                stack.append((c, ci))
            else:
                for x in leaves(kind, c):
                    clusters[ci]["leaving"].append((x, lam[e]))
    # stabilities: exact sums of the float64 terms, rounded once
    for C in clusters:
        total = Fraction(0)
        for _, lx in C["leaving"]:
            total += Fraction(lx - C["birth"])
        for di in C["children"]:
            D = clusters[di]
            total += D["size"] * Fraction(D["birth"] - C["birth"])
        C["stability"] = _round(total)
    # excess of mass, children before parents (creation order is top-down);
    # the root cluster is not a candidate
    selected = [False] * len(clusters)
    score = [Fraction(0)] * len(clusters)
    for ci in range(len(clusters) - 1, 0, -1):
        C = clusters[ci]
        if not C["children"]:
            selected[ci] = True
            score[ci] = Fraction(C["stability"])
            continue
        tot = sum((score[di] for di in C["children"]), Fraction(0))
        if Fraction(C["stability"]) >= tot:
            selected[ci] = True
            score[ci] = Fraction(C["stability"])
            st = list(C["children"])
            while st:
                d = st.pop()
                selected[d] = False
                st.extend(clusters[d]["children"])
        else:
            score[ci] = tot
    # labels: the one selected cluster on the path from a vertex's cluster up
    leave_cluster = np.full(n, -1, np.int64)
    for ci, C in enumerate(clusters):
        for x, _ in C["leaving"]:
            leave_cluster[x] = ci
    sel_anc = [-1] * len(clusters)
    for ci in range(1, len(clusters)):
        p = clusters[ci]["parent"]
        sel_anc[ci] = ci if selected[ci] else sel_anc[p]
    raw = [sel_anc[leave_cluster[x]] for x in range(n)]
    firsts = {}
    for x in range(n):
        if raw[x] >= 0 and raw[x] not in firsts:
            firsts[raw[x]] = x
    rank = {c: k for k, c in enumerate(sorted(firsts, key=lambda c: firsts[c]))}
    labels = np.array([rank[c] if c >= 0 else -1 for c in raw], np.int32)
    for ci, C in enumerate(clusters):
        C["selected"] = selected[ci]
        C["score"] = score[ci]
        C["label"] = rank.get(ci, -1)
        if members:
            C["members"] = sorted(leaves("e", C["edge"]))   # sizes >= mcs >= 2: edges
    return labels, {"clusters": clusters}
