"""Seeded synthetic tree generators shared by the tests and the benchmark.

This module only draws inputs: vertex ids, edge lists and fp32 weights.  It
holds none of the dendrogram arithmetic, so both the GPU path and the CPU
oracle can consume what it makes.  All randomness comes from numpy's PCG64
(``np.random.default_rng(seed)``).

Families (single trees have ``n`` vertices and ``m = n - 1`` edges):

* ``rrt``: random recursive tree, vertex i > 0 attaches to a parent drawn
  uniformly from [0, i); weights k * 2**-24 with k uniform in [1, 2**24),
  which are exact in fp32, lie in (0, 1) and repeat often at large m (ties are
  broken by edge index, so they are exercised on purpose).
* ``path_skewed``: a path with w_i = fp32(i + U(0, 0.5)) along it (computed in
  float64, rounded to nearest); its dendrogram has height ~n.
* ``star``, ``caterpillar``, ``binary``, ``path``: shapes for edge cases.

The canonical layout relabels vertices with a random permutation, shuffles
the edge order and flips each edge's orientation with probability 1/2, so no
locality is handed to the library for free.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

TWO_POW_M24 = 2.0 ** -24


@dataclass
class Tree:
    u: np.ndarray                 # int32[m]
    v: np.ndarray                 # int32[m]
    w: np.ndarray                 # float32[m]
    family: str = ""
    # for path trees: caller edge index of the k-th edge along the path and
    # the caller vertex id of the k-th path vertex
    path_eid: Optional[np.ndarray] = None
    path_vid: Optional[np.ndarray] = None
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.w.shape[0])

    @property
    def n(self) -> int:
        return self.m + 1


def uniform24(rng: np.random.Generator, m: int) -> np.ndarray:
    """fp32 weights k * 2**-24, k uniform in [1, 2**24): exact, in (0, 1)."""
    k = rng.integers(1, 1 << 24, size=m, dtype=np.int64)
    return (k.astype(np.float64) * TWO_POW_M24).astype(np.float32)


def _canonical(rng, child, parent, w, n, shuffle=True):
    """Relabel vertices, shuffle edges, flip orientations (see module doc)."""
    m = child.shape[0]
    if not shuffle:
        return (child.astype(np.int32), parent.astype(np.int32), w.astype(np.float32),
                np.arange(n, dtype=np.int64), np.arange(m, dtype=np.int64))
    vperm = rng.permutation(n).astype(np.int64)
    eperm = rng.permutation(m).astype(np.int64)          # new edge j = old edge eperm[j]
    flip = rng.random(m) < 0.5
    a = vperm[child[eperm]]
    b = vperm[parent[eperm]]
    u = np.where(flip, b, a).astype(np.int32)
    v = np.where(flip, a, b).astype(np.int32)
    return u, v, np.ascontiguousarray(w[eperm], dtype=np.float32), vperm, eperm


def rrt(n: int, seed: int, shuffle: bool = True, weights: Optional[np.ndarray] = None) -> Tree:
    """Random recursive tree on n vertices with uniform24 weights."""
    rng = np.random.default_rng(seed)
    if n < 1:
        raise ValueError("n >= 1")
    i = np.arange(1, n, dtype=np.int64)
    parent = np.floor(rng.random(n - 1) * i).astype(np.int64)
    np.minimum(parent, i - 1, out=parent)
    w = uniform24(rng, n - 1) if weights is None else np.asarray(weights, np.float32)
    u, v, w, _, _ = _canonical(rng, i, parent, w, n, shuffle)
    return Tree(u, v, w, family="rrt", meta=dict(n=n, seed=seed, shuffle=shuffle))


def _path_tree(rng, wpath: np.ndarray, n: int, shuffle: bool, family: str) -> Tree:
    m = n - 1
    child = np.arange(0, m, dtype=np.int64)
    parent = np.arange(1, n, dtype=np.int64)
    u, v, w, vperm, eperm = _canonical(rng, child, parent, wpath, n, shuffle)
    path_eid = np.empty(m, np.int64)
    path_eid[eperm] = np.arange(m, dtype=np.int64)
    return Tree(u, v, w, family=family, path_eid=path_eid.astype(np.int32),
                path_vid=vperm.astype(np.int32), meta=dict(n=n, shuffle=shuffle))


def path_skewed(n: int, seed: int, shuffle: bool = True) -> Tree:
    """Path with w_i = fp32(i + U(0, 0.5)) along it."""
    rng = np.random.default_rng(seed)
    m = n - 1
    wpath = (np.arange(m, dtype=np.float64) + 0.5 * rng.random(m)).astype(np.float32)
    t = _path_tree(rng, wpath, n, shuffle, "path_skewed")
    t.meta["seed"] = seed
    return t


def path(n: int, seed: int, kind: str = "random", shuffle: bool = True) -> Tree:
    """Path with sorted / reverse / random / equal uniform24 weights along it."""
    rng = np.random.default_rng(seed)
    m = n - 1
    wpath = uniform24(rng, m)
    if kind == "sorted":
        wpath = np.sort(wpath)
    elif kind == "reverse":
        wpath = np.sort(wpath)[::-1].copy()
    elif kind == "equal":
        wpath = np.full(m, 0.5, np.float32)
    elif kind != "random":
        raise ValueError(kind)
    return _path_tree(rng, wpath, n, shuffle, f"path_{kind}")


def star(n: int, seed: int, shuffle: bool = True) -> Tree:
    rng = np.random.default_rng(seed)
    i = np.arange(1, n, dtype=np.int64)
    u, v, w, vperm, _ = _canonical(rng, i, np.zeros(n - 1, np.int64), uniform24(rng, n - 1), n,
                                   shuffle)
    return Tree(u, v, w, family="star", meta=dict(center=int(vperm[0]), n=n))


def caterpillar(n: int, seed: int, shuffle: bool = True) -> Tree:
    """A spine of ceil(n/2) vertices, every other vertex hangs off the spine."""
    rng = np.random.default_rng(seed)
    i = np.arange(1, n, dtype=np.int64)
    spine = (n + 1) // 2
    parent = np.where(i < spine, i - 1, i - spine)
    return Tree(*_canonical(rng, i, parent, uniform24(rng, n - 1), n, shuffle)[:3],
                family="caterpillar")


def binary(n: int, seed: int, shuffle: bool = True) -> Tree:
    """Complete binary tree in heap order."""
    rng = np.random.default_rng(seed)
    i = np.arange(1, n, dtype=np.int64)
    return Tree(*_canonical(rng, i, (i - 1) // 2, uniform24(rng, n - 1), n, shuffle)[:3],
                family="binary")


def with_weights(t: Tree, w: np.ndarray) -> Tree:
    return Tree(t.u, t.v, np.ascontiguousarray(w, np.float32), family=t.family + "+w",
                path_eid=t.path_eid, path_vid=t.path_vid, meta=dict(t.meta))


def prufer_trees(n: int):
    """Every labelled tree on n >= 2 vertices (Pruefer decoding), as (u, v)."""
    import itertools
    if n == 2:
        yield np.array([0], np.int32), np.array([1], np.int32)
        return
    for seq in itertools.product(range(n), repeat=n - 2):
        degree = [1] * n
        for x in seq:
            degree[x] += 1
        us, vs = [], []
        for x in seq:
            leaf = min(j for j in range(n) if degree[j] == 1)
            us.append(leaf)
            vs.append(x)
            degree[leaf] -= 1
            degree[x] -= 1
        rest = [j for j in range(n) if degree[j] == 1]
        us.append(rest[0])
        vs.append(rest[1])
        yield np.array(us, np.int32), np.array(vs, np.int32)


@dataclass
class Batch:
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    edge_offsets: np.ndarray      # int64[T+1]
    families: list

    @property
    def n_trees(self) -> int:
        return int(self.edge_offsets.shape[0]) - 1

    @property
    def m(self) -> int:
        return int(self.edge_offsets[-1])

    def tree(self, t: int) -> Tree:
        e0, e1 = int(self.edge_offsets[t]), int(self.edge_offsets[t + 1])
        return Tree(self.u[e0:e1], self.v[e0:e1], self.w[e0:e1], family=self.families[t])


def log_uniform_sizes(rng, count: int, lo: int, hi: int) -> np.ndarray:
    x = np.exp(rng.uniform(np.log(lo), np.log(hi), size=count))
    return np.clip(np.rint(x).astype(np.int64), lo, hi)


def batch_sizes(n_trees: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """The vertex counts `batch` draws for these arguments (without building
    the trees), e.g. to shard a batch before generating it."""
    return log_uniform_sizes(np.random.default_rng(seed), n_trees, lo, hi)


def batch(n_trees: int, lo: int, hi: int, seed: int, families=("rrt", "path_skewed"),
          sizes: Optional[np.ndarray] = None, only: Optional[np.ndarray] = None) -> Batch:
    """Trees of log-uniform vertex counts in [lo, hi], family by a fair coin.
    With `only`, just those trees of the same batch are built, in that order
    (every tree has its own seed, so a subset equals the full batch's trees)."""
    rng = np.random.default_rng(seed)
    if sizes is None:
        sizes = log_uniform_sizes(rng, n_trees, lo, hi)
    fam_idx = rng.integers(0, len(families), size=n_trees)
    seeds = rng.integers(0, 2**62, size=n_trees)
    picked = range(n_trees) if only is None else [int(t) for t in only]
    us, vs, ws, fams = [], [], [], []
    offsets = np.zeros(len(picked) + 1, np.int64)
    for j, t in enumerate(picked):
        fam = families[int(fam_idx[t])]
        n = int(sizes[t])
        tr = rrt(n, int(seeds[t])) if fam == "rrt" else path_skewed(n, int(seeds[t]))
        us.append(tr.u)
        vs.append(tr.v)
        ws.append(tr.w)
        fams.append(fam)
        offsets[j + 1] = offsets[j] + tr.m
    cat = (lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt))
    return Batch(cat(us, np.int32), cat(vs, np.int32), cat(ws, np.float32), offsets, fams)


# ---------------------------------------------------------------------------
# HDBSCAN-shaped trees: mutual-reachability MSTs of Gaussian-mixture points
# ---------------------------------------------------------------------------
def gmm_points(n_points: int, seed: int, dim: int = 3, n_comp: int = 32) -> np.ndarray:
    """Points of an isotropic Gaussian mixture: means uniform in [0, 10]^dim,
    scales log-uniform in [0.01, 1], mixing weights ~ Dirichlet(1)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(0.0, 10.0, size=(n_comp, dim))
    scales = np.exp(rng.uniform(np.log(0.01), np.log(1.0), size=n_comp))
    mix = rng.dirichlet(np.ones(n_comp))
    comp = rng.choice(n_comp, size=n_points, p=mix)
    return means[comp] + rng.standard_normal((n_points, dim)) * scales[comp, None]


def core_distances(points: np.ndarray, min_pts: int) -> np.ndarray:
    """Distance to the min_pts-th nearest point, counting the point itself."""
    from scipy.spatial import cKDTree
    d, _ = cKDTree(points).query(points, k=min_pts, workers=-1)
    return d[:, -1] if min_pts > 1 else np.zeros(len(points))


def mr_mst_bruteforce(points: np.ndarray, min_pts: int):
    """Exact mutual-reachability MST by Prim's algorithm, O(n^2) (small n)."""
    n = len(points)
    core = core_distances(points, min_pts)
    in_tree = np.zeros(n, bool)
    best = np.full(n, np.inf)
    link = np.full(n, -1)
    best[0] = 0.0
    us, vs, ws = [], [], []
    for _ in range(n):
        cand = np.where(in_tree, np.inf, best)
        x = int(np.argmin(cand))
        in_tree[x] = True
        if link[x] >= 0:
            us.append(link[x])
            vs.append(x)
            ws.append(best[x])
        d = np.sqrt(((points - points[x]) ** 2).sum(axis=1))
        mr = np.maximum(np.maximum(core, core[x]), d)
        upd = (~in_tree) & (mr < best)
        best[upd] = mr[upd]
        link[upd] = x
    return np.array(us), np.array(vs), np.array(ws)


def mr_knn_mst(points: np.ndarray, min_pts: int, k: int = 32):
    """Spanning tree of the mutual-reachability graph restricted to k nearest
    neighbours.

    Weights are max(core(p), core(q), |p - q|) (core counts the point itself,
    minPts-th neighbour).  The minimum spanning forest of the symmetric k-NN
    graph (scipy) is computed first; its components are then joined, Boruvka
    style, by the lightest mutual-reachability edge between each point of a
    component and its k nearest points of every other component (kd-tree
    queries).
    On mixtures of well separated clusters this is the exact mutual-
    reachability MST except where a lighter non-k-NN edge exists, which the
    generator does not search for; ``mr_mst_bruteforce`` is the exact O(n^2)
    construction for small n.
    """
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components, minimum_spanning_tree
    from scipy.spatial import cKDTree
    n = len(points)
    kk = min(k, n - 1)
    tree = cKDTree(points)
    d, idx = tree.query(points, k=kk + 1, workers=-1)
    core = d[:, min_pts - 1] if min_pts > 1 else np.zeros(n)
    rows = np.repeat(np.arange(n), kk)
    cols = idx[:, 1:].reshape(-1)
    dd = d[:, 1:].reshape(-1)
    w = np.maximum(np.maximum(core[rows], core[cols]), dd)
    # symmetric: keep each pair once with its weight
    lo, hi = np.minimum(rows, cols), np.maximum(rows, cols)
    key = lo.astype(np.int64) * n + hi
    key, first = np.unique(key, return_index=True)
    g = coo_matrix((w[first] + 1e-300, (lo[first], hi[first])), shape=(n, n)).tocsr()
    f = minimum_spanning_tree(g).tocoo()
    us, vs, ws = list(f.row), list(f.col), list(f.data - 1e-300)
    n_comp, label = connected_components(coo_matrix((np.ones(len(us)), (us, vs)), shape=(n, n)),
                                         directed=False)
    while n_comp > 1:
        groups = [np.nonzero(label == c)[0] for c in range(n_comp)]
        trees = [cKDTree(points[g]) for g in groups]
        best = []   # per component: (weight, p, q)
        for c, gc in enumerate(groups):
            bw, bp, bq = np.inf, -1, -1
            for e, ge in enumerate(groups):
                if e == c:
                    continue
                kq = min(k, len(ge))
                dq, iq = trees[e].query(points[gc], k=kq, workers=-1)
                if kq == 1:
                    dq, iq = dq[:, None], iq[:, None]
                q = ge[iq]
                mr = np.maximum(np.maximum(core[gc][:, None], core[q]), dq)
                flat = int(np.argmin(mr))
                jp, jq = divmod(flat, kq)
                if mr[jp, jq] < bw:
                    bw, bp, bq = float(mr[jp, jq]), int(gc[jp]), int(q[jp, jq])
            best.append((bw, bp, bq))
        parent = np.arange(n_comp)

        def root(x):
            while parent[x] != x:
                parent[x] = parent[parent[x]]
                x = parent[x]
            return x
        for bw, bp, bq in sorted(best):
            a, b = root(label[bp]), root(label[bq])
            if a != b:
                parent[max(a, b)] = min(a, b)
                us.append(bp)
                vs.append(bq)
                ws.append(bw)
        comp_root = np.array([root(c) for c in range(n_comp)])
        _, label = np.unique(comp_root[label], return_inverse=True)
        n_comp = int(label.max()) + 1
    return np.array(us, np.int64), np.array(vs, np.int64), np.array(ws)


def hdbscan_tree(n_points: int, seed: int, min_pts: int = 16, method: str = "knn") -> Tree:
    """Mutual-reachability spanning tree (minPts counts the point itself) of
    n_points 3-D Gaussian-mixture points, fp32 weights, canonical layout.
    method "knn": ``mr_knn_mst``; "bruteforce": the exact MST (small n)."""
    pts = gmm_points(n_points, seed)
    if method == "bruteforce":
        a, b, w = mr_mst_bruteforce(pts, min_pts)
    else:
        a, b, w = mr_knn_mst(pts, min_pts)
    rng = np.random.default_rng(seed + 1)
    u, v, w32, _, _ = _canonical(rng, a.astype(np.int64), b.astype(np.int64),
                                 w.astype(np.float32), n_points, True)
    return Tree(u, v, w32, family="hdbscan", meta=dict(n_points=n_points, min_pts=min_pts,
                                                       seed=seed))
