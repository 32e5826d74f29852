"""The host-buffer entry point (pandora_dendrogram_host): host arrays in, host
arrays out, copies overlapped with the path; every element against the oracle."""
import os

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


def _host(pd, t, pinned):
    u, v, w = (torch.from_numpy(np.ascontiguousarray(x)) for x in (t.u, t.v, t.w))
    if pinned:
        u, v, w = u.pin_memory(), v.pin_memory(), w.pin_memory()
    ep, vp = pd.dendrogram_host(u, v, w)
    assert ep.device.type == "cpu" and vp.device.type == "cpu"
    return ep.numpy(), vp.numpy()


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("case", ["empty", "one_edge", "small_3000", "rrt_1e4", "rrt_1e6",
                                  "path_2e5", "star_5e4"])
def test_host_matches_oracle(pd, case, pinned):
    t = {"empty": lambda: inputs.rrt(1, 1),
         "one_edge": lambda: inputs.rrt(2, 2),
         "small_3000": lambda: inputs.rrt(3001, 3),
         "rrt_1e4": lambda: inputs.rrt(10_000, 0),
         "rrt_1e6": lambda: inputs.rrt(1_000_000, 5),
         "path_2e5": lambda: inputs.path_skewed(200_001, 6),
         "star_5e4": lambda: inputs.star(50_000, 7)}[case]()
    ep, vp = _host(pd, t, pinned)
    oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)


def test_host_errors_and_recovery(pd):
    t = inputs.rrt(20_000, 9)
    w = t.w.copy()
    w[1234] = np.nan
    with pytest.raises(pd.PandoraError) as ei:
        pd.dendrogram_host(torch.from_numpy(t.u), torch.from_numpy(t.v), torch.from_numpy(w))
    assert ei.value.code == 2
    ep, vp = _host(pd, t, True)
    oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
    np.testing.assert_array_equal(ep, oep)
    np.testing.assert_array_equal(vp, ovp)


def test_host_rejects_device_tensors(pd):
    t = inputs.rrt(100, 1)
    with pytest.raises(ValueError):
        pd.dendrogram_host(torch.from_numpy(t.u).cuda(), torch.from_numpy(t.v),
                           torch.from_numpy(t.w))


def test_host_above_bucketed_link_threshold(pd):
    """4*10^7 edges (above 2^25): the link stores edge_parent by caller-id
    buckets, and the host entry point copies edge_parent back range by range
    as the apply pass finishes each range of buckets; the endpoints arrive in
    chunks that the first sort pass takes one by one.  Every element against
    the oracle."""
    t = inputs.rrt(40_000_001, 8)
    ep, vp = _host(pd, t, pinned=True)
    oep, ovp = oracle.dendrogram_threads(t.u, t.v, t.w, os.cpu_count() or 1)
    np.testing.assert_array_equal(vp, ovp)
    np.testing.assert_array_equal(ep, oep)
