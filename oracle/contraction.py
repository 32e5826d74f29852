"""Plain numpy model of the paper's recursive alpha-edge contraction.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  It restates the steps
of the method in the paper's order, one level at a time, with no blocking or
fusion, so that per-level quantities of the GPU path (edges per level, alpha
counts) can be checked, and so that the method itself is checked against the
plain Kruskal oracle (the tests require ``dendrogram_by_contraction`` to equal
``oracle.dendrogram`` on every input they draw).

Steps and the passages they follow:

* ranks: edges sorted by (weight, caller index) ascending, Section 3.1; the
  paper sorts descending and calls the lightest edge the one with the highest
  index, so its maxI(v) is the minimum ascending rank here.
* Eq. 1: the parent of a vertex is its lightest incident edge.
* Eq. 2: an edge is an alpha-edge when it is the lightest incident edge of
  neither endpoint; leaf edges are the lightest at both endpoints, chain edges
  at exactly one (Section 3.1, types of edge nodes).
* Section 3.2: contract every non-alpha edge (connected components of the
  non-alpha edges), keep the vertex -> supervertex map, recurse on the tree of
  alpha-edges until a level has no alpha-edge.
* Section 3.3.2: an edge contracted at level l starts at the supervertex S
  that contains it at level l+1; at each level k = l+1, ... it belongs to the
  leaf chain hanging from p = P_k(S) (the lightest edge at S on level k) when
  it is lighter than p, otherwise S moves to its supervertex at level k+1.
  Edges never placed go to the root chain.  A chain is identified by its head
  edge p and by the endpoint of p that S is (the examples name chains "2L",
  "13R").
* Section 3.3.3: within a chain sorted by rank, each edge's parent is the next
  heavier one; the heaviest edge of a chain hangs from the chain's head edge,
  and the heaviest edge of the root chain is the root.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

from . import edge_order

ROOT = -1


def _components(n, a, b):
    if a.size == 0:
        return n, np.arange(n, dtype=np.int64)
    g = coo_matrix((np.ones(a.size, np.int8), (a, b)), shape=(n, n))
    return connected_components(g, directed=False)


def contraction_levels(u, v, w):
    """Per-level structures of the multilevel contraction.

    Returns (order, levels) where ``order[r]`` is the caller index of the edge
    of rank r and each level is a dict with the level's edges (``a``, ``b``:
    endpoints as level vertex ids, ``r``: global ranks, ascending), ``n``
    (vertices), ``min_inc`` (local index of the lightest incident edge of each
    vertex), ``alpha``/``leaf`` flags, and ``vmap`` (vertex -> supervertex of
    the next level).
    """
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    m = int(u.size)
    order = edge_order(w).astype(np.int64)
    a = u[order]
    b = v[order]
    r = np.arange(m, dtype=np.int64)
    n = m + 1
    levels = []
    while r.size > 0:
        ml = r.size
        min_inc = np.full(n, np.iinfo(np.int64).max, np.int64)
        local = np.arange(ml, dtype=np.int64)
        np.minimum.at(min_inc, a, local)
        np.minimum.at(min_inc, b, local)
        is_a = min_inc[a] == local
        is_b = min_inc[b] == local
        alpha = ~is_a & ~is_b
        leaf = is_a & is_b
        n_next, vmap = _components(n, a[~alpha], b[~alpha])
        levels.append(dict(a=a, b=b, r=r, n=n, min_inc=min_inc, alpha=alpha, leaf=leaf,
                           vmap=np.asarray(vmap, np.int64), n_next=int(n_next)))
        if not alpha.any():
            break
        a = np.asarray(vmap, np.int64)[a[alpha]]
        b = np.asarray(vmap, np.int64)[b[alpha]]
        r = r[alpha]
        n = int(n_next)
    return order, levels


def level_sizes(u, v, w):
    """Edges per contraction level: [m_0, m_1, ...] (m_0 = all edges)."""
    _, levels = contraction_levels(u, v, w)
    return [int(lv["r"].size) for lv in levels]


def chain_keys(u, v, w):
    """Chain of every edge by rank: (head rank, side) or (ROOT, 0)."""
    order, levels = contraction_levels(u, v, w)
    m = order.size
    head = np.full(m, ROOT, np.int64)
    side = np.zeros(m, np.int64)
    L = len(levels)
    for l0, lv in enumerate(levels):
        nonalpha = ~lv["alpha"]
        for i in np.nonzero(nonalpha)[0]:
            r = int(lv["r"][i])
            s = int(lv["vmap"][lv["a"][i]])
            for k in range(l0 + 1, L):
                up = levels[k]
                j = int(up["min_inc"][s])      # local index of P_k(S)
                p = int(up["r"][j])
                if r < p:
                    head[r] = p
                    side[r] = 1 if int(up["b"][j]) == s else 0
                    break
                s = int(up["vmap"][s])
    return order, head, side


def dendrogram_by_contraction(u, v, w):
    """Dendrogram by the method's own steps; must equal the Kruskal oracle."""
    order, head, side = chain_keys(u, v, w)
    m = order.size
    edge_parent = np.empty(m, np.int64)
    chains = {}
    for r in range(m):                       # ascending rank keeps chains sorted
        chains.setdefault((int(head[r]), int(side[r])), []).append(r)
    for (h, _), members in chains.items():
        for lo, hi in zip(members[:-1], members[1:]):
            edge_parent[order[lo]] = order[hi]
        edge_parent[order[members[-1]]] = -1 if h == ROOT else order[h]
    vertex_parent = np.full(m + 1, -1, np.int64)
    if m > 0:
        vertex_parent[:] = order[contraction_levels_first_min(u, v, order)]
    return edge_parent.astype(np.int32), vertex_parent.astype(np.int32)


def contraction_levels_first_min(u, v, order):
    """Rank of the lightest incident edge of every vertex (Eq. 1)."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    m = order.size
    rank = np.empty(m, np.int64)
    rank[order] = np.arange(m)
    best = np.full(m + 1, np.iinfo(np.int64).max, np.int64)
    np.minimum.at(best, u, rank)
    np.minimum.at(best, v, rank)
    return best
