"""The server's scheduling decisions (host logic, no GPU): lane choice and
admission by batch limits and HBM footprint."""
from collections import deque
from dataclasses import dataclass

from paper_2401_06089_gb300 import serving


@dataclass
class _Req:
    rid: int
    n_edges: int

    @property
    def m(self):
        return self.n_edges


def _server(budget=1 << 40, max_edges=1_000_000, max_trees=8, streams=3, cutoff=4096):
    s = object.__new__(serving.DendrogramServer)   # no CUDA streams: decisions only
    s.budget = budget
    s.max_batch_edges = max_edges
    s.max_batch_trees = max_trees
    s.free_streams = deque(range(streams))
    s.pending = deque()
    s.pending_small = deque()
    s.inflight = []
    s.bytes_in_use = 0
    s.small_cutoff = cutoff
    return s


def test_small_lane_first_and_last_stream_reserved():
    s = _server()
    s.pending.append(_Req(0, 100_000))
    s.pending_small.append(_Req(1, 100))
    assert s._pick_lane() is s.pending_small
    s.pending_small.clear()
    assert s._pick_lane() is s.pending           # three free streams
    s.free_streams = deque([0])
    s.inflight = ["a batch"]
    assert s._pick_lane() is None                # the last stream stays for small requests
    s.inflight = []
    assert s._pick_lane() is s.pending           # nothing running: no reason to wait
    s.small_cutoff = -1                          # one lane only
    s.inflight = ["a batch"]
    assert s._pick_lane() is s.pending


def test_admission_limits():
    s = _server(max_edges=250_000, max_trees=3)
    for i, m in enumerate([100_000, 100_000, 100_000, 10]):
        s.pending.append(_Req(i, m))
    got = s._take(s.pending)
    assert [r.rid for r in got] == [0, 1]        # a third would pass max_batch_edges
    s.pending.extendleft(reversed(got))
    s.max_batch_edges = 10**9
    got = s._take(s.pending)
    assert [r.rid for r in got] == [0, 1, 2]     # max_batch_trees
    s.pending.extendleft(reversed(got))
    # the HBM budget: only what fits next to the batches in flight
    one = serving.batch_footprint(100_000, 1)
    s.budget = one + 1
    got = s._take(s.pending)
    assert [r.rid for r in got] == [0]
    s.bytes_in_use = s.budget
    s.pending.appendleft(got[0])
    assert s._take(s.pending) == []


def test_footprint_grows_with_edges_and_trees():
    a = serving.batch_footprint(1_000_000, 1)
    assert serving.batch_footprint(2_000_000, 1) > a
    assert serving.batch_footprint(1_000_000, 100) > a
