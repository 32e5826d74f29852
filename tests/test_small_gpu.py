"""Parity of the single-block small-tree solver and of the batched dispatch.

Trees of at most 4096 edges can be solved by one thread block that keeps every
step of the method in shared memory.  These cases run the same seeded inputs
through that solver (each block size and layout capacity), through the
multi-kernel pipeline (solver switched off) and through the oracle, and
compare all three element by element.
"""
import numpy as np
import pytest

import oracle
from paper_2401_06089_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SIZES = [0, 1, 2, 3, 5, 31, 32, 33, 127, 128, 255, 256, 257, 511, 1000, 1023, 1024, 1025,
         2047, 2048, 3000, 4095, 4096]


@pytest.fixture(scope="module")
def pd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_06089_gb300 as pd
    pd.load_library()
    return pd


@pytest.fixture
def tuning(pd):
    saved = pd.get_tuning()
    yield pd
    pd.set_tuning(saved["small_max_edges"], saved["small_threads"], saved["split_min_permille"])


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(pd, t):
    ep, vp = pd.dendrogram(_dev(t.u), _dev(t.v), _dev(t.w))
    return ep.cpu().numpy(), vp.cpu().numpy()


def _tree(fam, m, seed):
    n = m + 1
    if fam == "rrt":
        return inputs.rrt(n, seed)
    if fam == "path":
        return inputs.path(max(n, 2), seed, kind="random") if m >= 1 else inputs.rrt(1, seed)
    if fam == "star":
        return inputs.star(max(n, 2), seed) if m >= 1 else inputs.rrt(1, seed)
    if fam == "ties":
        t = inputs.rrt(n, seed)
        rng = np.random.default_rng(seed)
        return inputs.with_weights(t, rng.integers(0, 3, size=t.m).astype(np.float32))
    raise ValueError(fam)


@pytest.mark.parametrize("threads", [256, 512, 1024])
@pytest.mark.parametrize("fam", ["rrt", "path", "star", "ties"])
def test_single_tree_all_sizes(tuning, fam, threads):
    pd = tuning
    for m in SIZES:
        t = _tree(fam, m, seed=m + 17)
        oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
        pd.set_tuning(4096, [threads] * 13)
        ep, vp = _run(pd, t)
        np.testing.assert_array_equal(vp, ovp, err_msg=f"{fam} m={m}")
        np.testing.assert_array_equal(ep, oep, err_msg=f"{fam} m={m}")
        pd.set_tuning(0)
        pep, pvp = _run(pd, t)
        np.testing.assert_array_equal(pep, oep, err_msg=f"pipeline {fam} m={m}")
        np.testing.assert_array_equal(pvp, ovp, err_msg=f"pipeline {fam} m={m}")


def test_special_floats_small(tuning):
    pd = tuning
    vals = np.array([-np.inf, -3.5, -1e-45, -0.0, 0.0, 1e-45, 1.17549435e-38, 0.5, 3e38,
                     np.inf], np.float32)
    rng = np.random.default_rng(19)
    for m in (1, 6, 99, 1500, 4096):
        t = inputs.rrt(m + 1, seed=m)
        t = inputs.with_weights(t, rng.choice(vals, size=t.m))
        oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
        ep, vp = _run(pd, t)
        np.testing.assert_array_equal(ep, oep)
        np.testing.assert_array_equal(vp, ovp)


def test_cutoff_boundary(tuning):
    """m at the cutoff goes to the solver, m one above to the pipeline; both exact."""
    pd = tuning
    pd.set_tuning(700)
    for m in (699, 700, 701):
        t = inputs.rrt(m + 1, seed=m)
        oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
        pd.profile_start()
        ep, vp = _run(pd, t)
        prof = pd.profile_read()
        np.testing.assert_array_equal(ep, oep)
        np.testing.assert_array_equal(vp, ovp)
        assert (prof["small_tree"]["launches"] == 1) == (m <= 700)
        assert (prof["mark"]["launches"] > 0) == (m > 700)


def _expect_error(pd, u, v, w, code):
    with pytest.raises(pd.PandoraError) as ei:
        pd.dendrogram(_dev(np.asarray(u, np.int32)), _dev(np.asarray(v, np.int32)),
                      _dev(np.asarray(w, np.float32)))
    assert ei.value.code == code


def test_errors_small(tuning):
    pd = tuning
    pd.set_tuning(4096)
    _expect_error(pd, [0, 1], [1, 2], [1.0, np.nan], 2)
    _expect_error(pd, [0, 1], [1, 3], [1.0, 2.0], 3)
    _expect_error(pd, [0, 1], [1, 1], [1.0, 2.0], 4)
    _expect_error(pd, [0, 1], [1, 0], [1.0, 2.0], 5)
    _expect_error(pd, [0, 1, 2], [1, 2, 0], [1.0, 2.0, 3.0], 5)
    # a cycle inside a larger small tree
    t = inputs.rrt(3001, seed=5)
    u = t.u.copy()
    u[100] = t.v[2000] if t.v[2000] != t.v[100] else t.u[2000]
    st, _, _ = oracle.dendrogram(u, t.v, t.w, check=False)
    if st == oracle.ERR_NOT_A_TREE:
        _expect_error(pd, u, t.v, t.w, 5)
    t = inputs.rrt(1001, seed=6)
    oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
    ep, vp = _run(pd, t)
    np.testing.assert_array_equal(ep, oep)


def _run_batched(pd, b):
    ep, vp = pd.dendrogram_batched(_dev(b.u), _dev(b.v), _dev(b.w), _dev(b.edge_offsets))
    return ep.cpu().numpy(), vp.cpu().numpy()


@pytest.mark.parametrize("cutoff", [0, 64, 700, 4096])
def test_batched_dispatch(tuning, cutoff):
    """Mixed sizes around every bucket edge and the cutoff; large trees go
    through the packed forest, small ones one block each."""
    pd = tuning
    pd.set_tuning(cutoff, [256, 512, 1024, 256, 512, 1024, 256, 512, 1024, 256, 512, 1024, 512])
    rng = np.random.default_rng(cutoff)
    sizes = np.array([1, 1, 2, 3, 9, 64, 65, 66, 255, 256, 700, 701, 702, 1023, 4096, 4097,
                      5000, 20_000, 1, 130], np.int64)   # vertices per tree
    sizes = sizes[rng.permutation(len(sizes))]
    b = inputs.batch(len(sizes), 1, 1, seed=cutoff + 1, sizes=sizes)
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    ep, vp = _run_batched(pd, b)
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)


def test_batched_dispatch_log_uniform(tuning):
    """The batched benchmark's size mix, scaled down: 512 trees of 2..200,000 vertices."""
    pd = tuning
    b = inputs.batch(512, 2, 200_000, seed=4)
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    for cutoff in (0, 4096):
        pd.set_tuning(cutoff)
        ep, vp = _run_batched(pd, b)
        np.testing.assert_array_equal(vp, ovp)
        np.testing.assert_array_equal(ep, oep)


def test_batched_dispatch_errors(tuning):
    """An error in a small tree and in a large tree of one batch both surface."""
    pd = tuning
    pd.set_tuning(4096)
    for bad in (1, 3):
        sizes = np.array([10, 5000, 20, 9000], np.int64)
        b = inputs.batch(len(sizes), 1, 1, seed=bad, sizes=sizes)
        w = b.w.copy()
        e0 = int(b.edge_offsets[bad])
        w[e0 + 2] = np.nan
        with pytest.raises(pd.PandoraError) as ei:
            pd.dendrogram_batched(_dev(b.u), _dev(b.v), _dev(w), _dev(b.edge_offsets))
        assert ei.value.code == 2
    # and the library keeps working
    b = inputs.batch(8, 2, 3000, seed=9)
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    ep, vp = _run_batched(pd, b)
    np.testing.assert_array_equal(ep, oep)
    np.testing.assert_array_equal(vp, ovp)


def test_async_small_tree_graph(tuning):
    """The single-tree asynchronous call takes the solver and can be captured."""
    pd = tuning
    pd.set_tuning(4096)
    t = inputs.rrt(3001, seed=21)
    oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
    u, v, w = _dev(t.u), _dev(t.v), _dev(t.w)
    ws = torch.empty(pd.workspace_size(t.m), dtype=torch.uint8, device="cuda")
    ep = torch.empty(t.m, dtype=torch.int32, device="cuda")
    vp = torch.empty(t.m + 1, dtype=torch.int32, device="cuda")
    pd.dendrogram_async(u, v, w, ws, (ep, vp))   # eager first (one-time attributes)
    torch.cuda.synchronize()
    assert pd.workspace_status(ws) == 0
    ep.fill_(-7)
    vp.fill_(-7)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pd.dendrogram_async(u, v, w, ws, (ep, vp))
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    assert pd.workspace_status(ws) == 0
    np.testing.assert_array_equal(ep.cpu().numpy(), oep)
    np.testing.assert_array_equal(vp.cpu().numpy(), ovp)


def _planned(pd, b, host_off=None):
    u, v, w, off = _dev(b.u), _dev(b.v), _dev(b.w), _dev(b.edge_offsets)
    ws = torch.empty(pd.workspace_size(b.m, b.n_trees), dtype=torch.uint8, device="cuda")
    ep = torch.empty(b.m, dtype=torch.int32, device="cuda")
    vp = torch.empty(b.m + b.n_trees, dtype=torch.int32, device="cuda")
    h = b.edge_offsets if host_off is None else host_off
    pd.dendrogram_batched_planned(u, v, w, off, h, ws, (ep, vp))
    st = pd.workspace_status(ws, raise_on_error=False)
    return st, ep.cpu().numpy(), vp.cpu().numpy()


@pytest.mark.parametrize("permille", [0, 50, 1000])
@pytest.mark.parametrize("cutoff", [0, 300, 4096])
def test_planned_matches_oracle(tuning, cutoff, permille):
    """Planned (asynchronous, host offsets) batched calls: split or not, equal
    to the oracle on a mix around the cutoff and the bucket edges."""
    pd = tuning
    pd.set_tuning(cutoff, None, permille)
    sizes = np.array([1, 2, 3, 40, 299, 300, 301, 302, 1025, 4096, 4097, 4098, 12_000, 1, 9],
                     np.int64)
    b = inputs.batch(len(sizes), 1, 1, seed=cutoff + permille, sizes=sizes)
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    st, ep, vp = _planned(pd, b)
    assert st == 0
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)


def test_planned_all_small_and_profile(tuning):
    """A batch of small trees only: no pipeline kernel runs, one solver launch
    per occupied size bucket."""
    pd = tuning
    pd.set_tuning(4096, None, 50)
    rng = np.random.default_rng(8)
    sizes = rng.integers(1, 4097, size=300).astype(np.int64)
    b = inputs.batch(len(sizes), 1, 1, seed=8, sizes=sizes)
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    pd.profile_start()
    st, ep, vp = _planned(pd, b)
    prof = pd.profile_read()
    assert st == 0
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)
    assert prof["mark"]["launches"] == 0
    buckets = {int(np.floor(np.log2(max(m, 1)))) for m in sizes - 1}
    assert prof["small_tree"]["launches"] == len(buckets)


def test_planned_graph_replay(tuning):
    """Capture one planned call (split batch) in a CUDA graph and replay it on
    new batches with the same tree sizes."""
    pd = tuning
    pd.set_tuning(4096, None, 0)
    sizes = inputs.log_uniform_sizes(np.random.default_rng(5), 200, 2, 30_000)
    batches = [inputs.batch(len(sizes), 0, 0, seed=s, sizes=sizes) for s in (41, 42, 43)]
    b0 = batches[0]
    u, v, w, off = _dev(b0.u), _dev(b0.v), _dev(b0.w), _dev(b0.edge_offsets)
    ws = torch.empty(pd.workspace_size(b0.m, b0.n_trees), dtype=torch.uint8, device="cuda")
    ep = torch.empty(b0.m, dtype=torch.int32, device="cuda")
    vp = torch.empty(b0.m + b0.n_trees, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pd.dendrogram_batched_planned(u, v, w, off, b0.edge_offsets, ws, (ep, vp))
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pd.dendrogram_batched_planned(u, v, w, off, b0.edge_offsets, ws, (ep, vp))
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


def test_planned_plan_mismatch_is_reported(tuning):
    """Host offsets that are a partition but not the device's: the device
    reports PANDORA_ERR_INVALID_ARGUMENT and the library keeps working."""
    pd = tuning
    pd.set_tuning(4096, None, 0)
    sizes = np.array([100, 9000, 50, 7000, 3000], np.int64)
    b = inputs.batch(len(sizes), 1, 1, seed=12, sizes=sizes)
    host = b.edge_offsets.copy()
    host[1] += 5000   # still a partition: tree 0 large and tree 1 small on the host
    st, _, _ = _planned(pd, b, host_off=host)
    assert st == 1
    st, ep, vp = _planned(pd, b)
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    assert st == 0
    np.testing.assert_array_equal(ep, oep)
    np.testing.assert_array_equal(vp, ovp)
