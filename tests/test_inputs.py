"""The seeded generators (CPU): determinism and the HDBSCAN-shaped recipe."""
import numpy as np
import pytest

import oracle
from paper_2401_06089_gb300 import inputs


def test_generators_are_seeded():
    a = inputs.rrt(1000, 5)
    b = inputs.rrt(1000, 5)
    assert np.array_equal(a.u, b.u) and np.array_equal(a.w, b.w)
    c = inputs.path_skewed(1000, 5)
    assert np.array_equal(np.sort(c.w), np.sort(inputs.path_skewed(1000, 5).w))


def test_uniform24_weights_are_exact_fp32_in_unit_interval():
    w = inputs.uniform24(np.random.default_rng(0), 100_000)
    assert w.dtype == np.float32 and (w > 0).all() and (w < 1).all()
    k = w.astype(np.float64) * 2.0 ** 24
    assert np.array_equal(k, np.round(k))


def test_core_distance_counts_the_point_itself():
    pts = inputs.gmm_points(400, 1)
    core = inputs.core_distances(pts, 16)
    d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    np.testing.assert_allclose(core, np.sort(d, axis=1)[:, 15])


def test_exact_mr_mst_matches_dense_scipy():
    from scipy.sparse.csgraph import minimum_spanning_tree
    pts = inputs.gmm_points(600, 2)
    core = inputs.core_distances(pts, 16)
    d = np.sqrt(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1))
    mr = np.maximum(np.maximum(core[:, None], core[None, :]), d)
    np.fill_diagonal(mr, 0.0)
    dense = minimum_spanning_tree(mr).data.sum()
    _, _, w = inputs.mr_mst_bruteforce(pts, 16)
    assert np.isclose(w.sum(), dense, rtol=1e-12)


@pytest.mark.parametrize("n", [2, 17, 3000])
def test_hdbscan_tree_is_a_spanning_tree(n):
    t = inputs.hdbscan_tree(n, seed=n, min_pts=min(16, n))
    assert t.m == n - 1
    ep, vp = oracle.dendrogram(t.u, t.v, t.w)   # raises unless it is a tree
    assert (ep == -1).sum() == 1


def test_increasing_path_construction_against_oracle():
    """The generator of the maximum-size test, at a small size on the CPU: its
    closed form holds for the oracle's dendrogram."""
    torch = pytest.importorskip("torch")
    import importlib.util, os
    spec = importlib.util.spec_from_file_location(
        "tpg", os.path.join(os.path.dirname(__file__), "test_parity_gpu.py"))
    tpg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(tpg)
    for m in (1, 2, 7, 1000, 65_537):
        u, v, w, pos = tpg.strictly_increasing_path(m, "cpu", a_mul=1_000_003)
        ep, vp = oracle.dendrogram(u.numpy(), v.numpy(), w.numpy())
        tpg.check_increasing_path(torch.from_numpy(ep), torch.from_numpy(vp), pos)
