"""Failure reporting of the bounded device loops, on a real GPU without
faulting or hanging it.

pandora_set_wait_report_limit makes the look-back waits and the union-find
loops record PANDORA_ERR_ITERATION_LIMIT once they run longer than a few
iterations, without cutting them short.  The input below has a long chain
of vertices whose lightest edges lead along it (weights increasing along the
first half of a path) next to many small components, so the contraction's
union-find runs on level 0 and takes more than one step: the status is set
on every call, deterministically.  The blocking call must report it, the
asynchronous call must leave it in the workspace with outputs that are
still exact (the loops were only reported, not cut), and the next call with
the default limit must be clean and bit-exact against the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2401_06089_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
ITERATION_LIMIT = 6


@pytest.fixture(scope="module")
def pd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_06089_gb300 as pd
    pd.load_library()
    return pd


def _chain_tree(n=1_000_000, seed=5):
    t = inputs.path(n, seed, kind="random")
    rng = np.random.default_rng(seed)
    w = np.empty(t.m, np.float32)
    half = t.m // 2
    w[t.path_eid[:half]] = np.arange(1, half + 1, dtype=np.float32)
    w[t.path_eid[half:]] = rng.integers(1, half, size=t.m - half).astype(np.float32)
    return inputs.with_weights(t, w)


def test_report_limit_sets_the_status_and_the_default_is_clean(pd):
    t = _chain_tree()
    dev = torch.device("cuda")
    u = torch.from_numpy(t.u).to(dev)
    v = torch.from_numpy(t.v).to(dev)
    w = torch.from_numpy(t.w).to(dev)
    oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
    pd.set_wait_report_limit(0)
    try:
        with pytest.raises(pd.PandoraError) as e:
            pd.dendrogram(u, v, w)
        assert e.value.code == ITERATION_LIMIT
        ws = torch.empty(pd.workspace_size(t.m), dtype=torch.uint8, device=dev)
        ep = torch.empty(t.m, dtype=torch.int32, device=dev)
        vp = torch.empty(t.m + 1, dtype=torch.int32, device=dev)
        pd.dendrogram_async(u, v, w, ws, (ep, vp))
        assert pd.workspace_status(ws, raise_on_error=False) == ITERATION_LIMIT
        np.testing.assert_array_equal(ep.cpu().numpy(), oep)
        np.testing.assert_array_equal(vp.cpu().numpy(), ovp)
    finally:
        pd.set_wait_report_limit(-1)
    gep, gvp = pd.dendrogram(u, v, w)
    np.testing.assert_array_equal(gep.cpu().numpy(), oep)
    np.testing.assert_array_equal(gvp.cpu().numpy(), ovp)
    pd.dendrogram_async(u, v, w, ws, (ep, vp))
    assert pd.workspace_status(ws, raise_on_error=False) == 0
