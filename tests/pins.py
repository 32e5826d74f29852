"""Independent restatements that pin the CPU oracle (pure Python / numpy).

None of these routines is used by the oracle or by the GPU path.  Each one
reaches the single-linkage dendrogram by a different route than the oracle's
Kruskal agglomeration, so a dropped term, a wrong tie rule or a transposed
endpoint in the oracle fails at least one of them:

* ``brute_force``: the definition read from Section 2.1 and Section 3.1:
  the parent of edge e is the lightest edge heavier than e that touches the
  cluster e belongs to once every edge not heavier than e has been merged;
  the parent of a vertex is its lightest incident edge (Eq. 1).
* ``top_down``: the divisive construction of Section 2.2.1 (remove the
  heaviest edge, its children are the heaviest edges of the two parts).
* ``lcda_check``: Theorem 1 (the lowest common dendrogram ancestor of two
  edges is the heaviest edge on the tree path joining them).
* ``check_invariants``: properties that hold at any size (one root at the
  heaviest edge, parents heavier than children, every edge node has exactly
  two children counting vertex nodes, Eq. 1 for vertices).
"""
from __future__ import annotations

import math
from collections import defaultdict

import numpy as np


def order_key(w, e):
    """Sort key of edge e: weight, then -0.0 before +0.0, then caller index."""
    x = float(w[e])
    neg_zero = (x == 0.0 and math.copysign(1.0, x) < 0)
    return (x, 0 if neg_zero else 1, int(e))


def ranks_numpy(w) -> np.ndarray:
    """rank[e] of every edge under the same order, via numpy's lexsort."""
    w = np.asarray(w, np.float32)
    m = w.shape[0]
    pos_zero = ~np.signbit(w)
    order = np.lexsort((np.arange(m), pos_zero, w.astype(np.float64)))
    rank = np.empty(m, np.int64)
    rank[order] = np.arange(m)
    return rank


def brute_force(u, v, w):
    u = [int(x) for x in u]
    v = [int(x) for x in v]
    m = len(u)
    n = m + 1
    keys = [order_key(w, e) for e in range(m)]
    incident = defaultdict(list)
    for e in range(m):
        incident[u[e]].append(e)
        incident[v[e]].append(e)
    edge_parent = [-1] * m
    for e in range(m):
        # cluster of e in the forest of edges not heavier than e
        allowed = {g for g in range(m) if keys[g] <= keys[e]}
        comp = {u[e], v[e]}
        stack = [u[e], v[e]]
        while stack:
            x = stack.pop()
            for g in incident[x]:
                if g in allowed:
                    for y in (u[g], v[g]):
                        if y not in comp:
                            comp.add(y)
                            stack.append(y)
        cands = [f for f in range(m) if keys[f] > keys[e] and (u[f] in comp or v[f] in comp)]
        edge_parent[e] = min(cands, key=lambda f: keys[f]) if cands else -1
    vertex_parent = []
    for x in range(n):
        inc = incident[x]
        vertex_parent.append(min(inc, key=lambda f: keys[f]) if inc else -1)
    return np.array(edge_parent, np.int32), np.array(vertex_parent, np.int32)


def top_down(u, v, w):
    u = [int(x) for x in u]
    v = [int(x) for x in v]
    m = len(u)
    n = m + 1
    keys = [order_key(w, e) for e in range(m)]
    edge_parent = [-2] * m
    vertex_parent = [-2] * n
    if m == 0:
        return np.array([], np.int32), np.array([-1], np.int32)

    def split(vertices, edges, parent):
        if not edges:
            (x,) = vertices
            vertex_parent[x] = parent
            return
        h = max(edges, key=lambda f: keys[f])
        edge_parent[h] = parent
        rest = [f for f in edges if f != h]
        adj = defaultdict(list)
        for f in rest:
            adj[u[f]].append(f)
            adj[v[f]].append(f)
        for root in (u[h], v[h]):
            seen = {root}
            stack = [root]
            while stack:
                x = stack.pop()
                for f in adj[x]:
                    for y in (u[f], v[f]):
                        if y not in seen:
                            seen.add(y)
                            stack.append(y)
            part_edges = [f for f in rest if u[f] in seen]
            split(seen, part_edges, h)

    split(set(range(n)), list(range(m)), -1)
    return np.array(edge_parent, np.int32), np.array(vertex_parent, np.int32)


def _ancestors(edge_parent, e):
    out = [e]
    while edge_parent[out[-1]] != -1:
        out.append(int(edge_parent[out[-1]]))
    return out


def lcda_check(u, v, w, edge_parent) -> None:
    """Theorem 1 for every pair of edges; raises AssertionError on a mismatch."""
    u = [int(x) for x in u]
    v = [int(x) for x in v]
    m = len(u)
    keys = [order_key(w, e) for e in range(m)]
    adj = defaultdict(list)
    for e in range(m):
        adj[u[e]].append((v[e], e))
        adj[v[e]].append((u[e], e))
    anc = [_ancestors(edge_parent, e) for e in range(m)]
    depth_of = [{a: k for k, a in enumerate(chain)} for chain in anc]
    for i in range(m):
        # edges on the vertex path from u[i] to every vertex (BFS tree)
        prev = {u[i]: (None, None)}
        queue = [u[i]]
        for x in queue:
            for y, e in adj[x]:
                if y not in prev:
                    prev[y] = (x, e)
                    queue.append(y)
        for j in range(i + 1, m):
            path = {i, j}
            x = u[j]
            while prev[x][0] is not None:
                path.add(prev[x][1])
                x = prev[x][0]
            heaviest = max(path, key=lambda f: keys[f])
            lca = next(a for a in anc[j] if a in depth_of[i])
            assert lca == heaviest, (i, j, lca, heaviest)


def check_invariants(u, v, w, edge_parent, vertex_parent) -> None:
    """Properties of any single-linkage dendrogram, checked with numpy."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    ep = np.asarray(edge_parent, np.int64)
    vp = np.asarray(vertex_parent, np.int64)
    m = u.shape[0]
    n = m + 1
    assert ep.shape == (m,) and vp.shape == (n,)
    if m == 0:
        assert vp[0] == -1
        return
    rank = ranks_numpy(w)
    roots = np.nonzero(ep == -1)[0]
    assert roots.size == 1, f"{roots.size} roots"
    assert rank[roots[0]] == m - 1, "root is not the heaviest edge"
    nonroot = ep != -1
    assert ((ep[nonroot] >= 0) & (ep[nonroot] < m)).all()
    assert (rank[ep[nonroot]] > rank[nonroot.nonzero()[0]]).all(), "parent lighter than child"
    assert ((vp >= 0) & (vp < m)).all()
    children = np.bincount(ep[nonroot], minlength=m) + np.bincount(vp, minlength=m)
    assert (children == 2).all(), "an edge node without exactly two children"
    # Eq. 1: vertex parent is incident and lightest among incident edges
    assert ((u[vp] == np.arange(n)) | (v[vp] == np.arange(n))).all(), "vertex parent not incident"
    best = np.full(n, np.iinfo(np.int64).max)
    np.minimum.at(best, u, rank)
    np.minimum.at(best, v, rank)
    assert (rank[vp] == best).all(), "vertex parent not the lightest incident edge"
