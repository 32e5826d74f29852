"""Pins of the flat-cluster oracle (oracle/flat.py).

* Clusters and stabilities against a brute force that never looks at the
  dendrogram: it removes the tree's edges from the heaviest down (ties: larger
  caller index first), follows the connected components with a graph search,
  and scores every cluster in the per-point form of the stability: the exact
  sum over its points of fl(lambda at which the point stops being in the
  cluster - lambda at the cluster's birth), rounded once.
* The selection against an exhaustive search: the selected clusters form a
  set of non-root clusters, no two on one root path, of largest total
  stability (every such set is enumerated); when the largest total is reached
  by one set only, it is that set.
* Labels from the selection and the member lists alone.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import flat
from paper_2401_06089_gb300 import inputs


def _components(n, edges, alive):
    adj = [[] for _ in range(n)]
    for k, (a, b) in enumerate(edges):
        if alive[k]:
            adj[a].append(b)
            adj[b].append(a)
    comp = [-1] * n
    for s in range(n):
        if comp[s] >= 0:
            continue
        comp[s] = s
        st = [s]
        while st:
            x = st.pop()
            for y in adj[x]:
                if comp[y] < 0:
                    comp[y] = s
                    st.append(y)
    return comp


def sweep_clusters(u, v, w, mcs):
    """Clusters of the component sweep: list of (members, birth, stability,
    parent index), the root first."""
    n = len(w) + 1
    edges = list(zip(u.tolist(), v.tolist()))
    order = sorted(range(len(w)), key=lambda k: (float(w[k]), k), reverse=True)
    alive = [True] * len(w)
    clusters = [{"points": frozenset(range(n)), "birth": 0.0, "parent": -1, "leave": {}}]
    where = {frozenset(range(n)): 0}   # live component -> cluster index
    for k in order:
        lam = 1.0 / float(np.float64(w[k]))
        a, b = edges[k]
        comp = _components(n, edges, alive)
        K = frozenset(x for x in range(n) if comp[x] == comp[a])
        alive[k] = False
        comp = _components(n, edges, alive)
        A = frozenset(x for x in K if comp[x] == comp[a])
        Bp = frozenset(x for x in K if comp[x] == comp[b])
        ci = where.pop(K, None)
        if ci is None:
            continue
        C = clusters[ci]
        if len(A) >= mcs and len(Bp) >= mcs:
            for x in K:
                C["leave"][x] = lam
            for part in (A, Bp):
                clusters.append({"points": part, "birth": lam, "parent": ci, "leave": {}})
                where[part] = len(clusters) - 1
        else:
            for part in (A, Bp):
                if len(part) >= mcs:
                    where[part] = ci
                else:
                    for x in part:
                        C["leave"][x] = lam
    out = []
    for C in clusters:
        total = sum((Fraction(l - C["birth"]) for l in C["leave"].values()), Fraction(0))
        out.append((C["points"], C["birth"], total.numerator / total.denominator, C["parent"]))
    return out


def antichains(children, c):
    """Every set of clusters in c's subtree with no two on one root path,
    the empty set included."""
    kids = children[c]
    below = [frozenset()]
    for d in kids:
        below = [a | b for a in below for b in antichains(children, d)]
    return below + [frozenset([c])]


def check_selection(info):
    cl = info["clusters"]
    children = [[] for _ in cl]
    for i, C in enumerate(cl):
        if C["parent"] >= 0:
            children[C["parent"]].append(i)
    cands = [frozenset()]
    for d in children[0]:
        cands = [a | b for a in cands for b in antichains(children, d)]
    value = {s: sum((Fraction(cl[i]["stability"]) for i in s), Fraction(0)) for s in cands}
    best = max(value.values())
    chosen = frozenset(i for i, C in enumerate(cl) if C["selected"])
    assert chosen in value, "selection has two clusters on one root path or the root"
    assert value[chosen] == best
    winners = [s for s in cands if value[s] == best]
    if len(winners) == 1:
        assert chosen == winners[0]


def labels_from(info, n):
    lab = -np.ones(n, np.int64)
    for i, C in enumerate(info["clusters"]):
        if C["selected"]:
            lab[C["members"]] = i
    out = -np.ones(n, np.int32)
    seen = {}
    for x in range(n):
        if lab[x] >= 0:
            out[x] = seen.setdefault(lab[x], len(seen))
    return out


@pytest.mark.parametrize("seed", range(48))
def test_oracle_matches_component_sweep(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 24))
    t = inputs.rrt(n, seed) if seed % 2 else inputs.path(max(n, 2), seed, kind="random")
    w = t.w
    if seed % 4 == 0:   # ties
        w = rng.integers(1, 4, size=t.m).astype(np.float32)
    elif seed % 4 == 2:  # wide dynamic range
        w = np.exp2(rng.uniform(-60, 60, size=t.m)).astype(np.float32)
    mcs = int(rng.integers(2, 6))
    ep, vp = oracle.dendrogram(t.u, t.v, w)
    labels, info = flat.hdbscan_labels(ep, vp, w, mcs, members=True)
    ref = sweep_clusters(t.u, t.v, w, mcs)
    got = sorted((tuple(C["members"]), C["birth"], C["stability"]) for C in info["clusters"])
    exp = sorted((tuple(sorted(p)), b, s) for p, b, s, _ in ref)
    assert got == exp
    check_selection(info)
    np.testing.assert_array_equal(labels, labels_from(info, t.n))


def test_two_separated_groups():
    """Two groups of 4 points, tight inside (weight 1), joined by one heavy
    edge (weight 10), plus a far outlier (weight 100): with mcs = 3 the two
    groups are the clusters and the outlier is noise."""
    u = np.array([0, 1, 2, 4, 5, 6, 3, 0], np.int32)
    v = np.array([1, 2, 3, 5, 6, 7, 4, 8], np.int32)
    w = np.array([1, 1, 1, 1, 1, 1, 10, 100], np.float32)
    ep, vp = oracle.dendrogram(u, v, w)
    labels, info = flat.hdbscan_labels(ep, vp, w, 3)
    np.testing.assert_array_equal(labels, [0, 0, 0, 0, 1, 1, 1, 1, -1])
    # each group: 4 points born at 1/10 and leaving at 1, four equal terms
    assert [C["stability"] for C in info["clusters"][1:]] == [4 * (1.0 - 0.1)] * 2


def test_two_pairs():
    """A 4-point path 0-1-2-3 with weights 1, 2, 1 and mcs = 2: the middle edge
    splits {0,1} and {2,3}, born at 1/2, each leaving at 1: stabilities
    2 * (1 - 1/2) = 1 each; they are the root's children, so both are selected."""
    u = np.array([0, 1, 2], np.int32)
    v = np.array([1, 2, 3], np.int32)
    w = np.array([1, 2, 1], np.float32)
    ep, vp = oracle.dendrogram(u, v, w)
    labels, info = flat.hdbscan_labels(ep, vp, w, 2)
    np.testing.assert_array_equal(labels, [0, 0, 1, 1])
    assert [C["stability"] for C in info["clusters"][1:]] == [1.0, 1.0]


def test_parent_wins_a_tie():
    """Tree 0-1 (1), 0-2 (2), 2-3 (1/4), 1-4 (1), 3-5 (1/4), 4-6 (1/2), mcs 2.
    Edge 0-2 (lambda 1/2) splits A = {0,1,4,6} and B = {2,3,5}.  In A, edge 1-4
    goes before 0-1 (equal weights, larger index first) at lambda 1 and splits
    {0,1} and {4,6}: stability(A) = 4 * (1 - 1/2) = 2; {0,1} leaves at once
    (stability 0), {4,6} at lambda 2 (stability 2 * (2 - 1) = 2).  A's
    stability equals its children's total, so A is kept.  B loses point 5 and
    then {2,3} at lambda 4: stability 3 * (4 - 1/2) = 10.5."""
    u = np.array([1, 2, 3, 4, 5, 6], np.int32)
    v = np.array([0, 0, 2, 1, 3, 4], np.int32)
    w = np.array([1, 2, 0.25, 1, 0.25, 0.5], np.float32)
    ep, vp = oracle.dendrogram(u, v, w)
    labels, info = flat.hdbscan_labels(ep, vp, w, 2, members=True)
    np.testing.assert_array_equal(labels, [0, 0, 1, 1, 0, 1, 0])
    got = sorted((C["members"], C["stability"], C["selected"]) for C in info["clusters"])
    assert got == [([0, 1], 0.0, False), ([0, 1, 2, 3, 4, 5, 6], 3.5, False),
                   ([0, 1, 4, 6], 2.0, True), ([2, 3, 5], 10.5, True), ([4, 6], 2.0, False)]


def test_too_small_for_any_cluster_is_all_noise():
    t = inputs.rrt(6, 1)
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    labels, info = flat.hdbscan_labels(ep, vp, t.w, 10)
    assert (labels == -1).all()
    assert not any(C["selected"] for C in info["clusters"])


def test_single_vertex():
    labels, _ = flat.hdbscan_labels(np.zeros(0, np.int32), np.zeros(1, np.int32),
                                    np.zeros(0, np.float32), 2)
    np.testing.assert_array_equal(labels, [-1])


def test_rejects_bad_arguments():
    t = inputs.rrt(5, 0)
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    with pytest.raises(ValueError):
        flat.hdbscan_labels(ep, vp, t.w, 1)
    w = t.w.copy()
    w[0] = 0.0
    with pytest.raises(ValueError):
        flat.hdbscan_labels(ep, vp, w, 2)


def test_invariants_on_a_larger_tree():
    t = inputs.hdbscan_tree(3000, seed=2, method="bruteforce")
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    for mcs in (5, 15, 50):
        labels, info = flat.hdbscan_labels(ep, vp, t.w, mcs)
        k = labels.max() + 1
        assert k >= 1
        counts = np.bincount(labels[labels >= 0], minlength=k)
        assert (counts >= mcs).all()
        firsts = [int(np.flatnonzero(labels == c)[0]) for c in range(k)]
        assert firsts == sorted(firsts)
        assert sum(C["selected"] for C in info["clusters"]) == k
        # every non-root cluster has exactly two children or none
        nkids = np.bincount([C["parent"] for C in info["clusters"][1:]],
                            minlength=len(info["clusters"]))
        assert set(nkids.tolist()) <= {0, 2}
