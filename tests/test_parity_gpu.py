"""Parity of the CUDA path with the CPU oracle (bit-exact: the outputs are ints).

Every case feeds the same seeded inputs to the library (through its C ABI,
via the ctypes binding) and to the oracle, and compares both output arrays
element by element.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import contraction
from paper_2401_06089_gb300 import inputs
import golden_io
import pins

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


def run_gpu(pd, t, **kw):
    out = pd.dendrogram(_dev(t.u), _dev(t.v), _dev(t.w), **kw)
    return tuple(x.cpu().numpy() if isinstance(x, torch.Tensor) else x for x in out)


def assert_parity(pd, t, **kw):
    ep, vp = run_gpu(pd, t, **kw)[:2]
    oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)
    return ep, vp


@pytest.mark.parametrize("path", golden_io.all_cases(), ids=os.path.basename)
def test_golden(pd, path):
    u, v, w, ep, vp = golden_io.load(path)
    t = inputs.Tree(u, v, w)
    gep, gvp = run_gpu(pd, t)
    np.testing.assert_array_equal(gep, ep)
    np.testing.assert_array_equal(gvp, vp)


@pytest.mark.parametrize("seed", range(10))
def test_rrt_1e4(pd, seed):
    """Random recursive tree, n = 10^4, uniform fp32 weights (parity seeds 0-9)."""
    assert_parity(pd, inputs.rrt(10_000, seed))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 31, 32, 33, 255, 257, 2047, 2048, 2049, 2050,
                               4095, 4096, 4097, 4098, 8193, 12289, 65537])
def test_sizes_across_tiles(pd, n):
    """Ragged tails around the 2048-vertex and 4096-key tiles."""
    assert_parity(pd, inputs.rrt(n, seed=n))
    if n >= 2:
        assert_parity(pd, inputs.path(n, seed=n, kind="random"))


@pytest.mark.parametrize("fam", ["star", "caterpillar", "binary"])
@pytest.mark.parametrize("n", [2, 3, 1000, 100_001])
def test_shapes(pd, fam, n):
    assert_parity(pd, getattr(inputs, fam)(n, seed=7))


@pytest.mark.parametrize("kind", ["sorted", "reverse", "random", "equal"])
def test_paths(pd, kind):
    assert_parity(pd, inputs.path(50_001, seed=3, kind=kind))


def test_path_skewed_small(pd):
    t = inputs.path_skewed(300_001, seed=2)
    ep, vp = assert_parity(pd, t)
    cep, cvpp = oracle.cartesian_path(t.w[t.path_eid], t.path_eid)
    np.testing.assert_array_equal(ep, cep)


def test_unshuffled_layout(pd):
    assert_parity(pd, inputs.rrt(200_000, seed=4, shuffle=False))
    assert_parity(pd, inputs.path_skewed(200_000, seed=4, shuffle=False))


@pytest.mark.parametrize("alphabet", [1, 2, 3, 16])
def test_heavy_ties(pd, alphabet):
    rng = np.random.default_rng(alphabet)
    t = inputs.rrt(100_000, seed=alphabet)
    t = inputs.with_weights(t, rng.integers(0, alphabet, size=t.m).astype(np.float32))
    assert_parity(pd, t)


def test_special_floats(pd):
    vals = np.array([-np.inf, -3.5, -1e-45, -0.0, 0.0, 1e-45, 1e-40, 1.17549435e-38, 0.5, 3e38,
                     np.inf], np.float32)
    rng = np.random.default_rng(9)
    for n in (2, 7, 100, 5000, 70_000):
        t = inputs.rrt(n, seed=n)
        t = inputs.with_weights(t, rng.choice(vals, size=t.m))
        assert_parity(pd, t)


def test_random_small_trees_bulk(pd):
    rng = np.random.default_rng(123)
    for _ in range(150):
        n = int(rng.integers(1, 300))
        fam = int(rng.integers(0, 3))
        t = (inputs.rrt(n, int(rng.integers(1 << 30))) if fam == 0 else
             inputs.path(max(n, 2), int(rng.integers(1 << 30))) if fam == 1 else
             inputs.star(max(n, 2), int(rng.integers(1 << 30))))
        if rng.random() < 0.5:
            t = inputs.with_weights(t, rng.integers(0, 4, size=t.m).astype(np.float32))
        assert_parity(pd, t)


def test_level_sizes_match_contraction_model(pd):
    """Per-level edge counts equal those of the numpy model of Section 3.2."""
    for t in (inputs.rrt(50_000, seed=1), inputs.path_skewed(40_000, seed=2),
              inputs.caterpillar(30_001, seed=3), inputs.star(5000, seed=4)):
        _, _, st = run_gpu(pd, t, stats=True)
        assert st["level_edges"] == contraction.level_sizes(t.u, t.v, t.w)
        assert st["n_levels"] <= int(np.ceil(np.log2(t.m + 1)))
        for me, nv in zip(st["level_edges"], st["level_vertices"]):
            assert nv == me + 1


def test_deterministic(pd):
    t = inputs.rrt(300_000, seed=8)
    a = run_gpu(pd, t)
    b = run_gpu(pd, t)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_workspace_and_pool_paths_agree(pd):
    t = inputs.rrt(100_000, seed=10)
    ws = torch.empty(pd.workspace_size(t.m), dtype=torch.uint8, device="cuda")
    a = run_gpu(pd, t, workspace=ws)
    b = run_gpu(pd, t)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_invariants_1e6(pd):
    t = inputs.rrt(1_000_000, seed=12)
    ep, vp = assert_parity(pd, t)
    pins.check_invariants(t.u, t.v, t.w, ep, vp)


def test_path_skewed_above_2pow24(pd):
    """Beyond 2**24 consecutive fp32 path weights tie; ties break by index."""
    t = inputs.path_skewed(20_000_000, seed=2)
    ep, vp = run_gpu(pd, t)
    cep, cvpp = oracle.cartesian_path(t.w[t.path_eid], t.path_eid)
    np.testing.assert_array_equal(ep, cep)
    np.testing.assert_array_equal(vp[t.path_vid], cvpp)


# ---- errors -------------------------------------------------------------------

def _expect_error(pd, u, v, w, code):
    with pytest.raises(pd.PandoraError) as ei:
        pd.dendrogram(_dev(np.asarray(u, np.int32)), _dev(np.asarray(v, np.int32)),
                      _dev(np.asarray(w, np.float32)))
    assert ei.value.code == code


def test_error_codes(pd):
    _expect_error(pd, [0, 1], [1, 2], [1.0, np.nan], 2)
    _expect_error(pd, [0, 1], [1, 3], [1.0, 2.0], 3)
    _expect_error(pd, [0, -1], [1, 2], [1.0, 2.0], 3)
    _expect_error(pd, [0, 1], [1, 1], [1.0, 2.0], 4)
    _expect_error(pd, [0, 1], [1, 0], [1.0, 2.0], 5)          # duplicate edge
    # a cycle 0-1-2-0 plus a cut-off vertex 3
    _expect_error(pd, [0, 1, 2], [1, 2, 0], [1.0, 2.0, 3.0], 5)
    rng = np.random.default_rng(5)
    t = inputs.rrt(10_000, seed=5)
    u = t.u.copy()
    u[123] = t.v[4567] if t.v[4567] != t.v[123] else t.u[4567]   # likely a cycle
    st, _, _ = oracle.dendrogram(u, t.v, t.w, check=False)
    if st == oracle.ERR_NOT_A_TREE:
        _expect_error(pd, u, t.v, t.w, 5)
    # the library still works after errors
    assert_parity(pd, inputs.rrt(1000, seed=1))


# ---- batched -----------------------------------------------------------------

def run_batched(pd, b, **kw):
    out = pd.dendrogram_batched(_dev(b.u), _dev(b.v), _dev(b.w), _dev(b.edge_offsets), **kw)
    return tuple(x.cpu().numpy() if isinstance(x, torch.Tensor) else x for x in out)


@pytest.mark.parametrize("seed", range(3))
def test_batched_matches_oracle(pd, seed):
    b = inputs.batch(200, 1, 20_000, seed=seed)
    ep, vp = run_batched(pd, b)[:2]
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)


def test_batched_tree_equals_single_call(pd):
    b = inputs.batch(20, 2, 5000, seed=11)
    ep, vp = run_batched(pd, b)[:2]
    for t in range(b.n_trees):
        e0, e1 = int(b.edge_offsets[t]), int(b.edge_offsets[t + 1])
        sep, svp = run_gpu(pd, b.tree(t))
        np.testing.assert_array_equal(ep[e0:e1], sep)
        np.testing.assert_array_equal(vp[e0 + t:e1 + t + 1], svp)


def test_batched_with_empty_trees(pd):
    sizes = np.array([1, 1, 2, 1, 3, 1000, 1, 2, 4097, 1], np.int64)
    b = inputs.batch(len(sizes), 1, 1, seed=3, sizes=sizes)
    ep, vp = run_batched(pd, b)[:2]
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)


def test_batched_bad_offsets(pd):
    b = inputs.batch(4, 10, 100, seed=1)
    off = b.edge_offsets.copy()
    off[-1] += 1
    with pytest.raises(pd.PandoraError) as ei:
        pd.dendrogram_batched(_dev(b.u), _dev(b.v), _dev(b.w), _dev(off[:-1]))
    assert ei.value.code in (1, 3, 5)
    off = b.edge_offsets.copy()
    off[1], off[2] = off[2], off[1]
    with pytest.raises(pd.PandoraError) as ei:
        pd.dendrogram_batched(_dev(b.u), _dev(b.v), _dev(b.w), _dev(off))
    assert ei.value.code == 1


def test_hdbscan_shaped_tree(pd):
    """Mutual-reachability spanning tree of 3-D Gaussian-mixture points with
    minPts = 16: many weights equal a core distance, so ties are common."""
    t = inputs.hdbscan_tree(200_000, seed=3)
    ep, vp = assert_parity(pd, t)
    pins.check_invariants(t.u, t.v, t.w, ep, vp)


@pytest.mark.parametrize("family", ["rrt", "path_skewed"])
def test_between_level0_and_level1_bucketing_thresholds(pd, family):
    """2*10^7 vertices: level 0 (above 2^24 vertices) marks by buckets with the
    flag pass while level 1 marks directly, and the chain keys (26 bits) take
    the three-pass 9 + 9 + 8-bit sort; every element against the oracle."""
    n = 20_000_000
    t = inputs.rrt(n, 5) if family == "rrt" else inputs.path_skewed(n, 6)
    assert_parity(pd, t)


# ---- full size, in the launch configuration bench.py times ---------------------

@pytest.mark.parametrize("family", ["rrt", "path_skewed"])
def test_full_size_1e8(pd, family):
    """n = 10^8 vertices, the benchmark's trees (seeds 1 and 2), called like
    bench.py (caller workspace, blocking entry point); every output element is
    compared with the oracle; the path also with its closed form."""
    n, seed = 100_000_000, (1 if family == "rrt" else 2)
    t = inputs.rrt(n, seed) if family == "rrt" else inputs.path_skewed(n, seed)
    ws = torch.empty(pd.workspace_size(t.m), dtype=torch.uint8, device="cuda")
    ep, vp = run_gpu(pd, t, workspace=ws)
    del ws
    torch.cuda.empty_cache()
    oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)
    if family == "path_skewed":
        cep, _ = oracle.cartesian_path(t.w[t.path_eid], t.path_eid)
        np.testing.assert_array_equal(ep, cep)


def test_batched_forest_above_bucketed_marking_threshold(pd):
    """A forest of 4.4*10^7 vertices: level 0 marks by vertex buckets (more
    than 2^24 vertices), across tree boundaries; every element against the
    oracle."""
    sizes = np.array([12_000_000, 3, 11_000_000, 1, 10_000_000, 11_000_000, 2], np.int64)
    b = inputs.batch(len(sizes), 1, 1, seed=17, sizes=sizes)
    ep, vp = run_batched(pd, b)[:2]
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)


def strictly_increasing_path(m, device, a_mul=1_000_000_007, b_add=12345):
    """A path of m edges whose weights strictly increase along it: path edge i
    gets the fp32 whose order key (the sort's sign-flip transform) is
    0x00800000 + i -- consecutive floats upward from -FLT_MAX, through
    -0.0 < +0.0 and the subnormals (finite for m <= 2^31 - 2).  Caller position
    c holds path edge (a_mul * c + b_add) mod m, an affine permutation, with a
    hashed orientation.  Returns (u, v, w, pos), pos[i] = caller position of
    path edge i; everything elementwise, so it runs on the device at any size."""
    import math
    assert math.gcd(a_mul, m) == 1
    c = torch.arange(m, dtype=torch.int64, device=device)
    order = (c * a_mul + b_add) % m
    flip = ((c * 0x9E3779B1) >> 16) & 1
    a = order.to(torch.int32)
    u = torch.where(flip == 1, a + 1, a)
    v = torch.where(flip == 1, a, a + 1)
    del flip, a
    k = order + 0x00800000
    bits = torch.where(k >= 2**31, k - 2**31, 0xFFFFFFFF - k)
    del k
    bits = torch.where(bits >= 2**31, bits - 2**32, bits).to(torch.int32)
    w = bits.view(torch.float32)
    del bits, order
    inv = pow(a_mul, -1, m)
    i = c   # reuse: c now plays the path index
    pos = (((i - b_add) % m) * inv % m).to(torch.int32)
    del c, i
    return u, v, w, pos


def check_increasing_path(ep, vp, pos):
    """Closed form of a path whose weights increase along it: path edge i hangs
    from path edge i + 1, the last is the root; vertex x's lightest edge is
    path edge x - 1 (edge 0 for vertex 0)."""
    assert torch.equal(ep[pos[:-1].long()], pos[1:])
    assert int(ep[pos[-1].long()]) == -1
    assert int(vp[0]) == int(pos[0])
    assert torch.equal(vp[1:], pos)


def test_maximum_size_path(pd):
    """The largest input the ABI takes: n_edges + 1 = INT32_MAX vertices
    (2^31 - 2 edges, about 210 GB on the device with the workspace), a path
    from `strictly_increasing_path` in shuffled order with random orientation;
    every element is checked against the closed form.  Generated and checked on
    the device to keep host memory small."""
    import time
    t_start = time.perf_counter()

    def mark(what):
        print(f"[max-size] {what}: {time.perf_counter() - t_start:.1f} s", flush=True)

    free, total = torch.cuda.mem_get_info()
    m = 2**31 - 2
    if free < 240 * 2**30:
        pytest.skip(f"needs about 240 GB free on the device ({free / 2**30:.0f} GB)")
    dev = torch.device("cuda")
    u, v, w, pos = strictly_increasing_path(m, dev)
    torch.cuda.empty_cache()
    torch.cuda.synchronize()
    mark("inputs built")
    ws = torch.empty(pd.workspace_size(m), dtype=torch.uint8, device=dev)
    ep = torch.empty(m, dtype=torch.int32, device=dev)
    vp = torch.empty(m + 1, dtype=torch.int32, device=dev)
    pd.dendrogram(u, v, w, workspace=ws, out=(ep, vp))
    torch.cuda.synchronize()
    mark("dendrogram")
    del ws, u, v, w
    torch.cuda.empty_cache()
    check_increasing_path(ep, vp, pos)
    mark("checked")


def test_path_in_order_increasing_weights(pd):
    """The union-find worst case for id-ordered hooking: a path labelled and
    listed in order with strictly increasing weights (every vertex's pointer
    chain runs to one end), 3*10^7 vertices; checked against the closed form
    (each edge hangs from the next one) and, on a prefix, the oracle."""
    m = 30_000_000
    u = np.arange(m, dtype=np.int32)
    v = u + 1
    w = np.arange(1, m + 1, dtype=np.uint32).view(np.float32)   # consecutive positive floats
    ep, vp = run_gpu(pd, inputs.Tree(u, v, w))
    np.testing.assert_array_equal(ep[:-1], np.arange(1, m, dtype=np.int32))
    assert ep[-1] == -1
    np.testing.assert_array_equal(vp[1:], np.arange(m, dtype=np.int32))
    assert vp[0] == 0
    t = inputs.Tree(u[:100_000], v[:100_000], w[:100_000])
    assert_parity(pd, t)
