"""Asynchronous (no host sync, graph-capturable) entry points against the oracle.

The async path enqueues the worst-case number of contraction levels and every
sort pass; these tests require its outputs to equal the oracle's (integers,
zero tolerance), also when the call is captured in a CUDA graph and replayed
on new inputs.
"""
import numpy as np
import pytest

import oracle
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _async_single(pd, t):
    ws = torch.empty(pd.workspace_size(t.m), dtype=torch.uint8, device="cuda")
    ep = torch.empty(t.m, dtype=torch.int32, device="cuda")
    vp = torch.empty(t.m + 1, dtype=torch.int32, device="cuda")
    pd.dendrogram_async(_dev(t.u), _dev(t.v), _dev(t.w), ws, (ep, vp))
    assert pd.workspace_status(ws) == 0
    return ep.cpu().numpy(), vp.cpu().numpy()


@pytest.mark.parametrize("maker", [
    lambda: inputs.rrt(1, 0), lambda: inputs.rrt(2, 0), lambda: inputs.rrt(3, 1),
    lambda: inputs.rrt(10_000, 3), lambda: inputs.rrt(300_001, 4),
    lambda: inputs.path_skewed(100_000, 5), lambda: inputs.star(20_000, 6),
    lambda: inputs.caterpillar(50_001, 7), lambda: inputs.binary(65_536, 8),
    lambda: inputs.path(4097, 9, kind="equal")])
def test_async_single_matches_oracle(pd, maker):
    t = maker()
    ep, vp = _async_single(pd, t)
    oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
    np.testing.assert_array_equal(ep, oep)
    np.testing.assert_array_equal(vp, ovp)


@pytest.mark.parametrize("seed", range(2))
def test_async_batched_matches_oracle(pd, seed):
    b = inputs.batch(300, 1, 30_000, seed=10 + seed)
    ws = torch.empty(pd.workspace_size(b.m, b.n_trees), dtype=torch.uint8, device="cuda")
    ep = torch.empty(b.m, dtype=torch.int32, device="cuda")
    vp = torch.empty(b.m + b.n_trees, dtype=torch.int32, device="cuda")
    pd.dendrogram_batched_async(_dev(b.u), _dev(b.v), _dev(b.w), _dev(b.edge_offsets), ws, (ep, vp))
    assert pd.workspace_status(ws) == 0
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    np.testing.assert_array_equal(ep.cpu().numpy(), oep)
    np.testing.assert_array_equal(vp.cpu().numpy(), ovp)


def test_async_reports_device_errors(pd):
    t = inputs.rrt(1000, 1)
    w = t.w.copy()
    w[17] = np.nan
    ws = torch.empty(pd.workspace_size(t.m), dtype=torch.uint8, device="cuda")
    ep = torch.empty(t.m, dtype=torch.int32, device="cuda")
    vp = torch.empty(t.m + 1, dtype=torch.int32, device="cuda")
    pd.dendrogram_async(_dev(t.u), _dev(t.v), _dev(w), ws, (ep, vp))
    assert pd.workspace_status(ws, raise_on_error=False) == 2
    # a duplicate edge: a cycle plus a cut-off vertex
    u = t.u.copy()
    v = t.v.copy()
    u[5], v[5] = t.u[6], t.v[6]
    pd.dendrogram_async(_dev(u), _dev(v), _dev(t.w), ws, (ep, vp))
    assert pd.workspace_status(ws, raise_on_error=False) == 5
    # and the workspace is fine afterwards
    pd.dendrogram_async(_dev(t.u), _dev(t.v), _dev(t.w), ws, (ep, vp))
    assert pd.workspace_status(ws) == 0
    oep, _ = oracle.dendrogram(t.u, t.v, t.w)
    np.testing.assert_array_equal(ep.cpu().numpy(), oep)


def test_graph_capture_and_replay(pd):
    """Capture one batched call in a CUDA graph; replay on two new batches of
    the same tree sizes; each replay equals the oracle."""
    sizes = inputs.log_uniform_sizes(np.random.default_rng(3), 64, 2, 20_000)
    batches = [inputs.batch(len(sizes), 0, 0, seed=s, sizes=sizes) for s in (31, 32, 33)]
    b0 = batches[0]
    u = _dev(b0.u)
    v = _dev(b0.v)
    w = _dev(b0.w)
    off = _dev(b0.edge_offsets)
    ws = torch.empty(pd.workspace_size(b0.m, b0.n_trees), dtype=torch.uint8, device="cuda")
    ep = torch.empty(b0.m, dtype=torch.int32, device="cuda")
    vp = torch.empty(b0.m + b0.n_trees, dtype=torch.int32, device="cuda")
    # warm up on a side stream (lazy module loading happens outside capture)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pd.dendrogram_batched_async(u, v, w, off, ws, (ep, vp))
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pd.dendrogram_batched_async(u, v, w, off, ws, (ep, vp))
    for b in batches[1:]:
        u.copy_(_dev(b.u))
        v.copy_(_dev(b.v))
        w.copy_(_dev(b.w))
        g.replay()
        torch.cuda.synchronize()
        assert pd.workspace_status(ws) == 0
        oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
        np.testing.assert_array_equal(ep.cpu().numpy(), oep)
        np.testing.assert_array_equal(vp.cpu().numpy(), ovp)


def test_async_above_bucketed_marking_threshold(pd):
    """An asynchronous call on 7*10^7 vertices: levels are enqueued for their
    worst-case sizes (level 1: m/2 + 1 vertices), so levels 0 and 1 both mark
    by buckets (more than 2^25 vertices each), the second with its records in
    the sort buffers; every element against the oracle."""
    t = inputs.rrt(70_000_000, 21)
    ep, vp = _async_single(pd, t)
    oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
    np.testing.assert_array_equal(ep, oep)
    np.testing.assert_array_equal(vp, ovp)
