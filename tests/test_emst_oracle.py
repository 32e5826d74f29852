"""Pins of the mutual-reachability MST oracle (oracle/emst.py).

Routes that share nothing with the oracle's arithmetic:
* core distances from exact squared distances (rational arithmetic) of
  integer or float coordinates, neighbours ranked exactly;
* the MST's sorted weights against scipy's minimum spanning tree of a weight
  matrix built with scipy's own distance routine (exactly for integer
  coordinates, where every squared distance is an exact integer and sqrt is
  correctly rounded on both sides);
* the minimum over every labelled spanning tree (Pruefer enumeration) for
  n <= 6, totals compared exactly;
* the closed form of points on a line with min_pts = 1 (consecutive pairs);
* the cut property of every tree edge (n <= 40).
"""
from fractions import Fraction
import math

import numpy as np
import pytest

from oracle import emst
from paper_2401_06089_gb300 import inputs


def _exact_sq(p, a, b):
    return sum((Fraction(float(x)) - Fraction(float(y))) ** 2 for x, y in zip(p[a], p[b]))


@pytest.mark.parametrize("seed", range(8))
def test_core_distances_exact_ranking(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 40))
    p = rng.integers(-50, 50, size=(n, 3)).astype(np.float64) if seed % 2 else \
        rng.standard_normal((n, 2)).astype(np.float32)
    for k in (1, 2, min(4, n), n):
        core = emst.core_distances(p, k)
        for a in range(n):
            sq = sorted(_exact_sq(p, a, b) for b in range(n))
            want = math.sqrt(sq[k - 1])
            assert core[a] == pytest.approx(want, rel=1e-14, abs=0)
            if seed % 2:                     # integers: exact square, exact sqrt
                assert core[a] == math.sqrt(int(sq[k - 1]))


def _scipy_mst_weights(p, k):
    from scipy.sparse.csgraph import minimum_spanning_tree
    from scipy.spatial.distance import cdist
    d = cdist(p, p)
    sq = np.sort(d, axis=1)
    core = sq[:, k - 1]
    m = np.maximum(np.maximum(core[:, None], core[None, :]), d)
    np.fill_diagonal(m, 0.0)
    t = minimum_spanning_tree(m).tocoo()
    return np.sort(t.data)


@pytest.mark.parametrize("seed", range(10))
def test_weights_match_scipy(seed):
    pytest.importorskip("scipy")
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(3, 200))
    if seed % 2:
        p = np.unique(rng.integers(0, 1000, size=(n, 3)), axis=0).astype(np.float64)
    else:
        p = inputs.gmm_points(n, seed)
    k = int(rng.integers(2, 8))
    k = min(k, len(p))
    u, v, w = emst.mr_emst(p, k)
    assert len(w) == len(p) - 1
    got = np.sort(w)
    want = _scipy_mst_weights(p, k)
    if seed % 2:
        np.testing.assert_array_equal(got, want)
    else:
        np.testing.assert_allclose(got, want, rtol=1e-14, atol=0)


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_minimum_over_all_spanning_trees(n):
    rng = np.random.default_rng(n)
    for trial in range(4):
        p = rng.integers(0, 20, size=(n, 2)).astype(np.float64)
        k = int(rng.integers(1, n + 1))
        core = [math.sqrt(sorted(_exact_sq(p, a, b) for b in range(n))[k - 1]) for a in range(n)]

        def mr(a, b):
            return max(core[a], core[b], math.sqrt(_exact_sq(p, a, b)))
        best = min(sum(Fraction(mr(int(a), int(b))) for a, b in zip(tu, tv))
                   for tu, tv in inputs.prufer_trees(n))
        u, v, w = emst.mr_emst(p, k)
        assert sum(Fraction(float(x)) for x in w) == best


def test_line_closed_form():
    """min_pts = 1 on a line: the MST joins neighbours in sorted order."""
    rng = np.random.default_rng(5)
    xs = rng.permutation(rng.choice(10_000, size=300, replace=False)).astype(np.float64)
    p = xs[:, None]
    u, v, w = emst.mr_emst(p, 1)
    order = np.argsort(xs)
    want = {frozenset((int(a), int(b))) for a, b in zip(order[:-1], order[1:])}
    assert {frozenset((int(a), int(b))) for a, b in zip(u, v)} == want


@pytest.mark.parametrize("seed", range(4))
def test_cut_property(seed):
    """Every tree edge is a lightest edge across the cut it defines."""
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(5, 40))
    p = rng.standard_normal((n, 3))
    k = int(rng.integers(1, 6))
    u, v, w = emst.mr_emst(p, k)
    core = [math.sqrt(sorted(_exact_sq(p, a, b) for b in range(n))[k - 1]) for a in range(n)]
    adj = [[] for _ in range(n)]
    for e, (a, b) in enumerate(zip(u, v)):
        adj[a].append((b, e))
        adj[b].append((a, e))
    for e, (a, b) in enumerate(zip(u, v)):
        side = {int(a)}
        st = [int(a)]
        while st:
            x = st.pop()
            for y, f in adj[x]:
                if f != e and y not in side:
                    side.add(y)
                    st.append(y)
        assert int(b) not in side
        cross = min(max(core[x], core[y], math.sqrt(_exact_sq(p, x, y)))
                    for x in side for y in range(n) if y not in side)
        assert w[e] <= cross * (1 + 1e-14)


def test_agrees_with_the_input_generator():
    """The generator's exact construction (different code) gives the same
    sorted weights on HDBSCAN-shaped points."""
    p = inputs.gmm_points(500, 3)
    _, _, w = emst.mr_emst(p, 16)
    _, _, w2 = inputs.mr_mst_bruteforce(p, 16)
    np.testing.assert_allclose(np.sort(w), np.sort(w2), rtol=1e-14, atol=0)


def test_rejects_bad_min_pts():
    p = np.zeros((3, 2))
    with pytest.raises(ValueError):
        emst.core_distances(p, 0)
    with pytest.raises(ValueError):
        emst.core_distances(p, 4)
