"""Parity of the GPU HDBSCAN* flat clusters (pandora_hdbscan_labels) with the
oracle (oracle/flat.py): labels element by element and the stability of every
kept cluster bit for bit (both sides sum exactly and round once)."""
import numpy as np
import pytest

import oracle
from oracle import flat
from paper_2401_06089_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BAD_WEIGHT = 11
NOT_A_DENDROGRAM = 12
INVALID_ARGUMENT = 1


@pytest.fixture(scope="module")
def pd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_06089_gb300 as pd
    pd.load_library()
    return pd


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_flat(pd, ep, vp, w, mcs):
    lab, stab = pd.hdbscan_labels(_dev(ep), _dev(vp), _dev(w), mcs, stability=True)
    return lab.cpu().numpy(), stab.cpu().numpy()


def oracle_flat(ep, vp, w, mcs):
    lab, info = flat.hdbscan_labels(ep, vp, w, mcs)
    kept = sorted((C for C in info["clusters"] if C["label"] >= 0), key=lambda C: C["label"])
    return lab, np.array([C["stability"] for C in kept], np.float64)


def assert_flat_parity(pd, ep, vp, w, mcs):
    lab, stab = gpu_flat(pd, ep, vp, w, mcs)
    olab, ostab = oracle_flat(ep, vp, w, mcs)
    np.testing.assert_array_equal(lab, olab)
    assert stab.shape == ostab.shape
    np.testing.assert_array_equal(stab.view(np.uint64), ostab.view(np.uint64))
    return lab


def _weights(rng, t, kind):
    if kind == "ties":
        return rng.integers(1, 4, size=t.m).astype(np.float32)
    if kind == "wide":
        return np.exp2(rng.uniform(-120, 120, size=t.m)).astype(np.float32)
    return t.w


@pytest.mark.parametrize("seed", range(40))
def test_small_trees(pd, seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 400))
    t = inputs.rrt(n, seed) if seed % 2 else inputs.path(n, seed, kind="random")
    w = _weights(rng, t, ("plain", "ties", "wide")[seed % 3])
    mcs = int(rng.integers(2, 9))
    ep, vp = oracle.dendrogram(t.u, t.v, w)
    assert_flat_parity(pd, ep, vp, w, mcs)


@pytest.mark.parametrize("n", [2047, 2048, 2049, 4096, 4097, 8193, 65537])
def test_scan_tile_boundaries(pd, n):
    t = inputs.rrt(n, n)
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    for mcs in (2, 3, 40):
        assert_flat_parity(pd, ep, vp, t.w, mcs)


def test_hdbscan_tree_from_gpu_dendrogram(pd):
    """The composed pipeline: HDBSCAN-shaped spanning tree, GPU dendrogram, GPU
    flat clusters; the oracle takes the same dendrogram."""
    t = inputs.hdbscan_tree(50_000, seed=4)
    ep, vp = (x.cpu().numpy() for x in pd.dendrogram(_dev(t.u), _dev(t.v), _dev(t.w)))
    for mcs in (5, 16, 100):
        lab = assert_flat_parity(pd, ep, vp, t.w, mcs)
        assert lab.max() >= 1


def test_million_point_random_tree(pd):
    t = inputs.rrt(1_000_000, 11)
    ep, vp = (x.cpu().numpy() for x in pd.dendrogram(_dev(t.u), _dev(t.v), _dev(t.w)))
    lab = assert_flat_parity(pd, ep, vp, t.w, 8)
    assert lab.max() > 1000


def test_deep_path(pd):
    """A path with increasing weights: the dendrogram is one chain of depth n,
    which the Euler tour and the pointer jumping must climb in log n rounds."""
    n = 200_000
    rng = np.random.default_rng(3)
    u = np.arange(n - 1, dtype=np.int32)
    v = u + 1
    w = np.sort(rng.uniform(1, 2, size=n - 1)).astype(np.float32)
    ep, vp = oracle.dendrogram(u, v, w)
    for mcs in (2, 1000):
        assert_flat_parity(pd, ep, vp, w, mcs)


def test_degenerate_inputs(pd):
    # one point: noise
    lab = pd.hdbscan_labels(_dev(np.zeros(0, np.int32)), _dev(np.full(1, -1, np.int32)),
                            _dev(np.zeros(0, np.float32)), 2)
    assert lab.cpu().tolist() == [-1]
    # fewer points than min_cluster_size: all noise
    t = inputs.rrt(7, 1)
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    lab, stab = gpu_flat(pd, ep, vp, t.w, 8)
    assert (lab == -1).all() and stab.size == 0
    # two points, mcs 2: the only split leaves singletons: all noise
    ep, vp = oracle.dendrogram(np.array([0], np.int32), np.array([1], np.int32),
                               np.array([1], np.float32))
    assert_flat_parity(pd, ep, vp, np.array([1], np.float32), 2)
    # a star with equal weights: every edge ties, the chain of ties decides
    n = 3000
    u = np.zeros(n - 1, np.int32)
    v = np.arange(1, n, dtype=np.int32)
    w = np.ones(n - 1, np.float32)
    ep, vp = oracle.dendrogram(u, v, w)
    for mcs in (2, 5):
        assert_flat_parity(pd, ep, vp, w, mcs)


def test_large_tree_properties(pd):
    """10^7 points (no oracle at this size): kept clusters hold at least mcs
    points, are numbered by their smallest point, and have positive
    stabilities; two calls agree bit for bit."""
    t = inputs.rrt(10_000_000, 12)
    u, v, w = _dev(t.u), _dev(t.v), _dev(t.w)
    ep, vp = pd.dendrogram(u, v, w)
    lab, stab = pd.hdbscan_labels(ep, vp, w, 32, stability=True)
    lab2, stab2 = pd.hdbscan_labels(ep, vp, w, 32, stability=True)
    assert torch.equal(lab, lab2) and torch.equal(stab, stab2)
    lab = lab.cpu().numpy()
    k = int(lab.max()) + 1
    assert k == stab.numel() and k > 100
    counts = np.bincount(lab[lab >= 0], minlength=k)
    assert (counts >= 32).all()
    firsts = np.full(k, np.iinfo(np.int64).max)
    np.minimum.at(firsts, lab[lab >= 0], np.flatnonzero(lab >= 0))
    assert (np.diff(firsts) > 0).all()
    assert (stab.cpu().numpy() > 0).all()


def _status(pd, ep, vp, w, mcs):
    try:
        pd.hdbscan_labels(_dev(ep), _dev(vp), _dev(w), mcs)
    except pd.PandoraError as e:
        return e.code
    return 0


def test_errors(pd):
    t = inputs.rrt(500, 2)
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)
    assert _status(pd, ep, vp, t.w, 2) == 0
    assert _status(pd, ep, vp, t.w, 1) == INVALID_ARGUMENT
    for bad in (0.0, -1.0, np.nan, np.inf):
        w = t.w.copy()
        w[7] = bad
        assert _status(pd, ep, vp, w, 4) == BAD_WEIGHT
    # a parent lighter than its child
    e = int(np.flatnonzero(ep >= 0)[0])
    w = t.w.copy()
    w[ep[e]] = w[e] / 2
    assert _status(pd, ep, vp, w, 4) == NOT_A_DENDROGRAM
    # a parent out of range, two roots, an edge with three children
    for mutate in ("range", "roots", "three"):
        ep2, vp2 = ep.copy(), vp.copy()
        if mutate == "range":
            vp2[3] = len(ep)
        elif mutate == "roots":
            ep2[e] = -1
        else:
            x = int(np.flatnonzero(vp2 != vp2[0])[0])
            vp2[x] = vp2[0]
        assert _status(pd, ep2, vp2, t.w, 4) == NOT_A_DENDROGRAM
    # the library is still usable after the errors
    assert_flat_parity(pd, ep, vp, t.w, 4)
