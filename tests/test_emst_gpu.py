"""GPU mutual-reachability minimum spanning tree (pandora_mr_emst) against
the float32 reading of the oracle (oracle/emst.py: mr_emst_f32,
core_sq_distances_f32).

Under the strict edge order (mr2, smaller id, larger id) the tree is unique,
so the GPU's edge set must equal the oracle's exactly, every weight must be
the float32 square root of the oracle's mr2 for that edge, and the squared
core distances must be equal bit for bit.  Larger inputs are checked by what
holds at any size: n - 1 edges that span the points, core distances of
sampled points by brute force, and the least edge at sampled points (an edge
of every minimum spanning tree, by the cut property) present in the tree.
"""
import numpy as np
import pytest

import oracle
from oracle import emst as oemst
from paper_2401_06089_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_06089_gb300 as pd
    pd.load_library()
    return pd


def _gpu(pd, p, k):
    t = torch.from_numpy(np.ascontiguousarray(p, np.float32)).cuda()
    u, v, w, cs = pd.mr_emst(t, k, core=True)
    return u.cpu().numpy(), v.cpu().numpy(), w.cpu().numpy(), cs.cpu().numpy()


def _check_exact(pd, p, k):
    p = np.ascontiguousarray(p, np.float32)
    u, v, w, cs = _gpu(pd, p, k)
    n = len(p)
    core2 = oemst.core_sq_distances_f32(p, k)
    np.testing.assert_array_equal(cs, core2)
    assert len(u) == n - 1
    ou, ov, ow2 = oemst.mr_emst_f32(p, k)
    want = {(min(a, b), max(a, b)): x for a, b, x in zip(ou.tolist(), ov.tolist(), ow2)}
    got = list(zip(u.tolist(), v.tolist()))
    assert all(a < b for a, b in got)
    assert set(got) == set(want)
    for (a, b), x in zip(got, w):
        assert x == np.sqrt(np.float32(want[(a, b)]))


def _cases():
    rng = np.random.default_rng(11)
    yield "two points", np.array([[0, 0, 0], [1, 2, 2]], np.float32), 1
    yield "three points", rng.standard_normal((3, 3)), 2
    yield "gmm 17", inputs.gmm_points(17, 1), 5
    yield "gmm 200", inputs.gmm_points(200, 2), 16
    yield "gmm 1500", inputs.gmm_points(1500, 3), 16
    yield "gmm 4000", inputs.gmm_points(4000, 4), 16
    yield "gmm 2500 k=1", inputs.gmm_points(2500, 5), 1
    yield "normal 3000 k=2", rng.standard_normal((3000, 3)), 2
    yield "integer grid 1200", rng.integers(0, 12, size=(1200, 3)), 8
    yield "duplicates", np.repeat(rng.standard_normal((60, 3)), 9, axis=0)[
        rng.permutation(540)], 4
    yield "identical", np.ones((64, 3), np.float32), 4
    yield "collinear", np.stack([rng.permutation(1000), np.zeros(1000), np.zeros(1000)], 1), 3
    yield "wide range", rng.standard_normal((800, 3)) * np.float32(1e6), 7
    yield "k = 32", inputs.gmm_points(900, 6), 32


@pytest.mark.parametrize("name,p,k", list(_cases()), ids=[c[0] for c in _cases()])
def test_emst_matches_the_float32_oracle(pd, name, p, k):
    _check_exact(pd, p, k)


def test_single_point(pd):
    u, v, w, cs = _gpu(pd, np.zeros((1, 3), np.float32), 1)
    assert len(u) == 0 and len(w) == 0 and cs.tolist() == [0.0]


def test_errors(pd):
    p = torch.zeros((10, 3), dtype=torch.float32, device="cuda")
    for k in (0, 11, 33):
        with pytest.raises(pd.PandoraError) as e:
            pd.mr_emst(p, k)
        assert e.value.code == 1
    bad = torch.randn((100, 3), device="cuda")
    bad[57, 1] = float("nan")
    with pytest.raises(pd.PandoraError) as e:
        pd.mr_emst(bad, 4)
    assert e.value.name == "PANDORA_ERR_BAD_POINT"
    bad[57, 1] = float("inf")
    with pytest.raises(pd.PandoraError) as e:
        pd.mr_emst(bad, 4)
    assert e.value.name == "PANDORA_ERR_BAD_POINT"


@pytest.mark.parametrize("n", [200_000, 2_000_000])
def test_large_tree_properties(pd, n):
    p = inputs.gmm_points(n, 9).astype(np.float32)
    k = 16
    u, v, w, cs = _gpu(pd, p, k)
    assert len(u) == n - 1
    # spanning: n - 1 unions, each joining two different sets
    par = np.arange(n)

    def find(x):
        while par[x] != x:
            par[x] = par[par[x]]
            x = par[x]
        return x
    for a, b in zip(u.tolist(), v.tolist()):
        ra, rb = find(a), find(b)
        assert ra != rb
        par[ra] = rb
    rng = np.random.default_rng(n)
    edges = set(zip(u.tolist(), v.tolist()))
    for q in rng.choice(n, size=24, replace=False).tolist():
        d2 = oemst.sq_distances_f32(p, q)
        assert cs[q] == np.partition(d2, k - 1)[k - 1]
        w2 = np.maximum(np.maximum(cs, cs[q]), d2)
        w2[q] = np.inf
        best = float(w2.min())
        cand = np.flatnonzero(w2 == best)
        lo = np.minimum(cand, q)
        hi = np.maximum(cand, q)
        j = np.lexsort((hi, lo))[0]
        assert (int(lo[j]), int(hi[j])) in edges
    # weights are the square roots of mr2 over the edges
    i = rng.choice(n - 1, size=1000, replace=False)
    d2 = np.array([oemst.sq_distances_f32(p[[a, b]], 0)[1] for a, b in zip(u[i], v[i])],
                  np.float32)
    mr2 = np.maximum(np.maximum(cs[u[i]], cs[v[i]]), d2)
    np.testing.assert_array_equal(w[i], np.sqrt(mr2))


def test_emst_then_dendrogram_and_flat_clusters(pd):
    """The HDBSCAN* pipeline on the GPU: tree, dendrogram, flat clusters; the
    dendrogram equal to the oracle's of the same tree."""
    p = inputs.gmm_points(20_000, 12).astype(np.float32)
    t = torch.from_numpy(p).cuda()
    u, v, w = pd.mr_emst(t, 16)
    ep, vp = pd.dendrogram(u, v, w)
    oep, ovp = oracle.dendrogram(u.cpu().numpy(), v.cpu().numpy(), w.cpu().numpy())
    np.testing.assert_array_equal(ep.cpu().numpy(), oep)
    np.testing.assert_array_equal(vp.cpu().numpy(), ovp)
    labels = pd.hdbscan_labels(ep, vp, w, 32).cpu().numpy()
    from oracle import flat
    olabels, _ = flat.hdbscan_labels(oep, ovp, w.cpu().numpy(), 32)
    np.testing.assert_array_equal(labels, olabels)
