"""Pins of the float32 reading of the mutual-reachability MST oracle
(oracle/emst.py: sq_distances_f32, core_sq_distances_f32, mr_emst_f32).

Routes that share nothing with the oracle's arithmetic:
* integer coordinates, where every float32 operation of the reading is exact:
  the sorted squared weights equal those of the float64 oracle (pinned in
  tests/test_emst_oracle.py) exactly;
* float32 scalars, one point pair at a time, in the operation order the
  reading fixes, for every weight the oracle reports;
* for n <= 6, the spanning tree that minimises the sum of 2^rank over its
  edges (rank in the (mr2, smaller id, larger id) order), found by
  enumerating every labelled spanning tree: the same edge set;
* the cut property of every tree edge under the strict total order.
"""
import itertools

import numpy as np
import pytest

from oracle import emst
from paper_2401_06089_gb300 import inputs


def _d2_scalar(p, a, b):
    acc = None
    for k in range(p.shape[1]):
        dk = np.float32(p[a, k]) - np.float32(p[b, k])
        sq = np.float32(dk * dk)
        acc = sq if acc is None else np.float32(acc + sq)
    return np.float32(acc)


def _core2_scalar(p, k):
    n = len(p)
    return [sorted(_d2_scalar(p, a, b) for b in range(n))[k - 1] for a in range(n)]


def _mr2(p, core2, a, b):
    return max(core2[a], core2[b], _d2_scalar(p, a, b))


def _key(p, core2, a, b):
    return (_mr2(p, core2, a, b), min(a, b), max(a, b))


@pytest.mark.parametrize("seed", range(8))
def test_integer_coordinates_match_float64_oracle(seed):
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(2, 250))
    p = rng.integers(-300, 300, size=(n, 3)).astype(np.float32)
    k = int(rng.integers(1, min(n, 17) + 1))
    _, _, w2 = emst.mr_emst_f32(p, k)
    _, _, w = emst.mr_emst(p.astype(np.float64), k)
    np.testing.assert_array_equal(np.sort(w2.astype(np.float64)), np.sort(np.rint(w * w)))


@pytest.mark.parametrize("seed", range(6))
def test_weights_and_core_distances_by_scalars(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(3, 40))
    p = (inputs.gmm_points(n, seed) if seed % 2 else rng.standard_normal((n, 3))).astype(
        np.float32)
    k = int(rng.integers(1, min(n, 8) + 1))
    core2 = _core2_scalar(p, k)
    np.testing.assert_array_equal(emst.core_sq_distances_f32(p, k), np.array(core2, np.float32))
    u, v, w2 = emst.mr_emst_f32(p, k)
    for a, b, x in zip(u, v, w2):
        assert x == _mr2(p, core2, int(a), int(b))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_minimum_over_all_spanning_trees(n):
    rng = np.random.default_rng(600 + n)
    for trial in range(6):
        # few distinct values: many ties, decided by the vertex ids
        p = rng.integers(0, 3, size=(n, 2)).astype(np.float32)
        k = int(rng.integers(1, n + 1))
        core2 = _core2_scalar(p, k)
        pairs = sorted(itertools.combinations(range(n), 2), key=lambda e: _key(p, core2, *e))
        rank = {e: r for r, e in enumerate(pairs)}
        best, best_set = None, None
        for tu, tv in inputs.prufer_trees(n):
            es = {(min(int(a), int(b)), max(int(a), int(b))) for a, b in zip(tu, tv)}
            cost = sum(1 << rank[e] for e in es)
            if best is None or cost < best:
                best, best_set = cost, es
        u, v, _ = emst.mr_emst_f32(p, k)
        got = {(min(int(a), int(b)), max(int(a), int(b))) for a, b in zip(u, v)}
        assert got == best_set


@pytest.mark.parametrize("seed", range(16))
def test_cut_property_under_the_total_order(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(5, 30))
    if seed % 4 == 3:
        p = rng.standard_normal((n, 3)).astype(np.float32)
    elif seed % 2:
        p = rng.integers(0, 6, size=(n, 3)).astype(np.float32)
    else:   # few distinct distances: ties decided by the vertex ids
        p = rng.integers(0, 3, size=(n, 2)).astype(np.float32)
    k = int(rng.integers(1, 6))
    core2 = _core2_scalar(p, k)
    u, v, _ = emst.mr_emst_f32(p, k)
    adj = [[] for _ in range(n)]
    for e, (a, b) in enumerate(zip(u, v)):
        adj[int(a)].append((int(b), e))
        adj[int(b)].append((int(a), e))
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
        least = min(_key(p, core2, x, y) for x in side for y in range(n) if y not in side)
        assert _key(p, core2, int(a), int(b)) == least
