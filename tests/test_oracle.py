"""Pins of the CPU oracle against facts that do not come from the oracle.

CPU only (no ``gpu`` marker).  See ``pins.py`` for the independent routes.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from oracle import contraction
from paper_2401_06089_gb300 import inputs
import golden_io
import pins


def _eq(a, b):
    np.testing.assert_array_equal(np.asarray(a), np.asarray(b))


@pytest.mark.parametrize("path", golden_io.all_cases(), ids=os.path.basename)
def test_golden(path):
    u, v, w, ep, vp = golden_io.load(path)
    got_ep, got_vp = oracle.dendrogram(u, v, w)
    _eq(got_ep, ep)
    _eq(got_vp, vp)


def _random_small(rng, n, alphabet):
    t = inputs.rrt(n, int(rng.integers(1 << 30)))
    if alphabet:
        w = rng.integers(0, alphabet, size=n - 1).astype(np.float32)
        t = inputs.with_weights(t, w)
    return t


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_and_top_down_random(seed):
    rng = np.random.default_rng(1000 + seed)
    for _ in range(40):
        n = int(rng.integers(1, 41))
        alphabet = int(rng.choice([0, 2, 3, 5]))
        t = _random_small(rng, n, alphabet)
        ep, vp = oracle.dendrogram(t.u, t.v, t.w)
        bep, bvp = pins.brute_force(t.u, t.v, t.w)
        _eq(ep, bep)
        _eq(vp, bvp)
        tep, tvp = pins.top_down(t.u, t.v, t.w)
        _eq(ep, tep)
        _eq(vp, tvp)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_exhaustive_small(n):
    """Every labelled tree on n vertices x every weight word over {0,1,2}."""
    m = n - 1
    words = list(itertools.product([0.0, 1.0, 2.0], repeat=m))
    rng = np.random.default_rng(n)
    for u, v in inputs.prufer_trees(n):
        for word in words:
            w = np.array(word, np.float32)
            ep, vp = oracle.dendrogram(u, v, w)
            bep, bvp = pins.brute_force(u, v, w)
            _eq(ep, bep)
            _eq(vp, bvp)
        # a random relabelling of the edge indices changes the tie order
        p = rng.permutation(m)
        w = np.array(words[len(words) // 2], np.float32)[p]
        ep, vp = oracle.dendrogram(u[p], v[p], w)
        bep, bvp = pins.brute_force(u[p], v[p], w)
        _eq(ep, bep)
        _eq(vp, bvp)


def test_exhaustive_six_vertices_sampled_words():
    rng = np.random.default_rng(6)
    for u, v in inputs.prufer_trees(6):
        w = rng.integers(0, 3, size=5).astype(np.float32)
        ep, vp = oracle.dendrogram(u, v, w)
        bep, bvp = pins.brute_force(u, v, w)
        _eq(ep, bep)
        _eq(vp, bvp)


@pytest.mark.parametrize("n", [2, 3, 17, 1000])
def test_star_closed_form(n):
    """Theorem 4: a star's dendrogram is its edges in sorted order."""
    t = inputs.star(n, seed=n)
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    rank = pins.ranks_numpy(t.w)
    order = np.argsort(rank)
    expect = np.empty(n - 1, np.int64)
    expect[order[:-1]] = order[1:]
    expect[order[-1]] = -1
    _eq(ep, expect)
    c = t.meta["center"]
    assert vp[c] == order[0]
    leaves = np.where(t.u == c, t.v, t.u)
    _eq(vp[leaves], np.arange(n - 1))


@pytest.mark.parametrize("kind", ["random", "sorted", "reverse", "equal"])
@pytest.mark.parametrize("n", [2, 3, 50, 20000])
def test_path_cartesian_closed_form(kind, n):
    """Theorem 1 on a path: the dendrogram is the max-Cartesian tree."""
    t = inputs.path(n, seed=n, kind=kind)
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    cep, cvpp = oracle.cartesian_path(t.w[t.path_eid], t.path_eid)
    _eq(ep, cep)
    _eq(vp[t.path_vid], cvpp)


def test_path_cartesian_agrees_with_brute_force():
    """The Cartesian closed form itself, on small paths with ties."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        n = int(rng.integers(2, 30))
        t = inputs.path(n, seed=int(rng.integers(1 << 30)))
        w = rng.integers(0, 4, size=n - 1).astype(np.float32)
        t = inputs.with_weights(t, w)
        cep, cvpp = oracle.cartesian_path(t.w[t.path_eid], t.path_eid)
        bep, bvp = pins.brute_force(t.u, t.v, t.w)
        _eq(cep, bep)
        _eq(cvpp, bvp[t.path_vid])


def test_path_skewed_family_cartesian():
    t = inputs.path_skewed(200001, seed=2)
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    cep, cvpp = oracle.cartesian_path(t.w[t.path_eid], t.path_eid)
    _eq(ep, cep)
    _eq(vp[t.path_vid], cvpp)


def test_all_equal_weights_is_index_order():
    """Equal weights are ordered by caller index: same as weights = index."""
    t = inputs.rrt(3000, seed=3)
    ep1, vp1 = oracle.dendrogram(t.u, t.v, np.full(t.m, 0.25, np.float32))
    ep2, vp2 = oracle.dendrogram(t.u, t.v, np.arange(t.m, dtype=np.float32))
    _eq(ep1, ep2)
    _eq(vp1, vp2)


@pytest.mark.parametrize("seed", range(3))
def test_lcda_theorem(seed):
    rng = np.random.default_rng(50 + seed)
    n = int(rng.integers(100, 201))
    t = _random_small(rng, n, int(rng.choice([0, 3])))
    ep, _ = oracle.dendrogram(t.u, t.v, t.w)
    pins.lcda_check(t.u, t.v, t.w, ep)


def test_invariants_large_rrt():
    t = inputs.rrt(200000, seed=11)
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    pins.check_invariants(t.u, t.v, t.w, ep, vp)


def test_special_floats():
    vals = np.array([-np.inf, -1.5, -0.0, 0.0, 1e-45, 1e-40, 1.17549435e-38, 1.0, 3e38, np.inf],
                    np.float32)
    rng = np.random.default_rng(12)
    for _ in range(200):
        n = int(rng.integers(2, 25))
        t = inputs.rrt(n, seed=int(rng.integers(1 << 30)))
        t = inputs.with_weights(t, rng.choice(vals, size=n - 1))
        ep, vp = oracle.dendrogram(t.u, t.v, t.w)
        bep, bvp = pins.brute_force(t.u, t.v, t.w)
        _eq(ep, bep)
        _eq(vp, bvp)


def test_negative_zero_before_positive_zero():
    order = oracle.edge_order(np.array([0.0, -0.0, 0.0, -0.0], np.float32))
    _eq(order, [1, 3, 0, 2])


def test_error_codes():
    u = np.array([0, 1], np.int32)
    v = np.array([1, 2], np.int32)
    st, _, _ = oracle.dendrogram(u, v, np.array([1.0, np.nan], np.float32), check=False)
    assert st == oracle.ERR_NAN_WEIGHT
    st, _, _ = oracle.dendrogram(u, np.array([1, 3], np.int32), np.ones(2, np.float32),
                                 check=False)
    assert st == oracle.ERR_VERTEX_OUT_OF_RANGE
    st, _, _ = oracle.dendrogram(u, np.array([1, 1], np.int32), np.ones(2, np.float32),
                                 check=False)
    assert st == oracle.ERR_SELF_LOOP
    # duplicate edge: three vertices, two copies of (0, 1): a cycle, vertex 2 cut off
    st, _, _ = oracle.dendrogram(np.array([0, 1], np.int32), np.array([1, 0], np.int32),
                                 np.ones(2, np.float32), check=False)
    assert st == oracle.ERR_NOT_A_TREE


def test_single_vertex_and_single_edge():
    ep, vp = oracle.dendrogram(np.zeros(0, np.int32), np.zeros(0, np.int32),
                               np.zeros(0, np.float32))
    assert ep.size == 0 and list(vp) == [-1]
    ep, vp = oracle.dendrogram(np.array([1], np.int32), np.array([0], np.int32),
                               np.array([2.0], np.float32))
    assert list(ep) == [-1] and list(vp) == [0, 0]


@pytest.mark.parametrize("threads", [2, 3, 8, 16])
def test_threaded_sort_mode_equals_single_thread(threads):
    """The all-core timing mode (edge sort on several threads) gives the same
    dendrogram as the single-threaded oracle: ties across run boundaries,
    signed zeros and a tree smaller than the thread count included."""
    cases = [inputs.rrt(50_000, 7), inputs.path(20_000, 3, kind="random"),
             inputs.star(5_000, 1), inputs.rrt(5, 2)]
    heavy = inputs.rrt(30_000, 9)
    cases.append(inputs.with_weights(heavy, (np.arange(heavy.m) % 7).astype(np.float32)))
    zeros = inputs.rrt(10_000, 4)
    cases.append(inputs.with_weights(
        zeros, np.where(np.arange(zeros.m) % 3 == 0, -0.0, 0.0).astype(np.float32)))
    for t in cases:
        a = oracle.dendrogram(t.u, t.v, t.w)
        b = oracle.dendrogram_threads(t.u, t.v, t.w, threads)
        _eq(a[0], b[0])
        _eq(a[1], b[1])


def test_batched_equals_per_tree():
    b = inputs.batch(12, 2, 3000, seed=4)
    ep, vp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    for t in range(b.n_trees):
        tr = b.tree(t)
        e0, e1 = int(b.edge_offsets[t]), int(b.edge_offsets[t + 1])
        tep, tvp = oracle.dendrogram(tr.u, tr.v, tr.w)
        _eq(ep[e0:e1], tep)
        _eq(vp[e0 + t:e1 + t + 1], tvp)


# --- the method's own steps (numpy model) against the oracle ----------------

@pytest.mark.parametrize("seed", range(4))
def test_contraction_model_equals_oracle(seed):
    rng = np.random.default_rng(300 + seed)
    for _ in range(25):
        n = int(rng.integers(1, 400))
        fam = rng.integers(0, 4)
        if fam == 0:
            t = _random_small(rng, n, int(rng.choice([0, 2, 7])))
        elif fam == 1:
            t = inputs.path(max(n, 2), seed=int(rng.integers(1 << 30)))
        elif fam == 2:
            t = inputs.caterpillar(max(n, 2), seed=int(rng.integers(1 << 30)))
        else:
            t = inputs.binary(max(n, 2), seed=int(rng.integers(1 << 30)))
        ep, vp = oracle.dendrogram(t.u, t.v, t.w)
        cep, cvp = contraction.dendrogram_by_contraction(t.u, t.v, t.w)
        _eq(cep, ep)
        _eq(cvp, vp)


@pytest.mark.parametrize("gen", ["rrt", "path_skewed", "caterpillar"])
def test_contraction_level_invariants(gen):
    """Section 4.2: n_alpha = n_leaf - 1, n_alpha <= (m-1)/2, levels bounded."""
    t = getattr(inputs, gen)(30001, seed=5)
    _, levels = contraction.contraction_levels(t.u, t.v, t.w)
    m = t.m
    assert len(levels) <= int(np.ceil(np.log2(m + 1)))
    for lv in levels:
        ml = lv["r"].size
        n_alpha = int(lv["alpha"].sum())
        n_leaf = int(lv["leaf"].sum())
        assert n_alpha == n_leaf - 1
        assert 2 * n_alpha <= ml - 1
        assert lv["n"] == ml + 1
        assert lv["n_next"] == n_alpha + 1
    assert not levels[-1]["alpha"].any()

