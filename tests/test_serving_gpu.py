"""Continuous-batching server: every request's result is the same alone and
in the mix (exact equality: the outputs are integers)."""
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


def test_results_identical_alone_and_in_the_mix(pd):
    from paper_2401_06089_gb300.serving import DendrogramServer, Request, run_trace, batch_footprint
    rng = np.random.default_rng(7)
    sizes = inputs.log_uniform_sizes(rng, 24, 1, 200_000)
    pool = []
    for k, n in enumerate(sizes):
        t = inputs.rrt(int(n), seed=100 + k) if k % 3 else inputs.path_skewed(max(int(n), 2), 100 + k)
        pool.append((t, torch.from_numpy(t.u).cuda(), torch.from_numpy(t.v).cuda(),
                     torch.from_numpy(t.w).cuda()))
    torch.cuda.synchronize()
    n_req = 80
    pick = rng.integers(0, len(pool), size=n_req)
    arrivals = np.cumsum(rng.exponential(2e-4, size=n_req)).tolist()
    reqs = [Request(i, pool[p][1], pool[p][2], pool[p][3]) for i, p in enumerate(pick)]
    # a budget that holds only a few of the largest trees at once forces
    # admission to wait for memory and splits the stream into many batches
    budget = 3 * batch_footprint(int(sizes.max()), 1)
    server = DendrogramServer(budget, max_batch_edges=400_000, max_batch_trees=16, n_streams=3)
    results = run_trace(server, reqs, arrivals)
    assert len(results) == n_req
    batches = {}
    for r in results:
        batches.setdefault(r.batch_id, []).append(r.rid)
    assert len(batches) > 1
    assert max(len(x) for x in batches.values()) > 1, "no request shared a batch"
    assert server.max_inflight >= 2, "batches never overlapped"
    alone = {}
    for r in sorted(results, key=lambda x: x.rid):
        p = int(pick[r.rid])
        if p not in alone:
            t, u, v, w = pool[p]
            alone[p] = [x.cpu().numpy() for x in pd.dendrogram(u, v, w)]
        np.testing.assert_array_equal(r.edge_parent.cpu().numpy(), alone[p][0])
        np.testing.assert_array_equal(r.vertex_parent.cpu().numpy(), alone[p][1])
    for p in list(alone)[:6]:
        t = pool[p][0]
        oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
        np.testing.assert_array_equal(alone[p][0], oep)
        np.testing.assert_array_equal(alone[p][1], ovp)
