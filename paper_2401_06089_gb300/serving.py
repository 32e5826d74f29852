"""Continuous-batching dendrogram server on one GPU.

Requests are trees that already live in device memory (for example MSTs
produced on the GPU).  The server keeps every in-flight batch's inputs,
scratch and outputs on the device and admits work by HBM footprint:

* ``submit`` queues a request in one of two FIFO lanes: small requests (at
  most the single-block solver's cutoff, see ``set_tuning``) and the rest;
* ``step`` first retires finished batches (CUDA event query), then, while a
  stream is free, packs the oldest pending requests of a lane into one
  forest -- as many as fit the batch limits and the remaining HBM budget --
  and enqueues ``pandora_dendrogram_batched_planned`` for it on that stream
  (the server knows every request's size, so the call needs no host
  synchronisation and a batch of small trees runs entirely in the
  single-block solver, one block per tree);
* the small lane goes first and large batches never hold the last free
  stream, so a small request does not wait behind a batch of large trees;
* batches on different streams overlap on the device, and requests that
  arrive while others run are admitted as soon as a stream and memory free up.

Each request's result is exactly the dendrogram of its own tree: the batched
entry point treats the batch as a forest of independent trees with
tree-local ids, so a request gives the same output alone and in any mix.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field
from typing import List, Optional

from . import _binding as B


@dataclass
class Request:
    rid: int
    u: "object"                  # int32 CUDA tensor [m]
    v: "object"                  # int32 CUDA tensor [m]
    w: "object"                  # float32 CUDA tensor [m]
    t_arrival: float = 0.0

    @property
    def m(self) -> int:
        return int(self.w.numel())


@dataclass
class Result:
    rid: int
    edge_parent: "object"        # int32 CUDA tensor [m] (view into the batch output)
    vertex_parent: "object"      # int32 CUDA tensor [m + 1]
    t_arrival: float
    t_admit: float
    t_done: float
    batch_id: int

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


@dataclass
class _Batch:
    bid: int
    reqs: List[Request]
    stream: "object"
    event: "object"
    ws: "object"
    ep: "object"
    vp: "object"
    offsets: List[int]
    footprint: int
    t_admit: float
    keep: list = field(default_factory=list)


def batch_footprint(total_edges: int, n_trees: int) -> int:
    """Device bytes one batch holds while in flight: packed inputs (12 B/edge),
    offsets, outputs (8 B/edge + 4 B/tree) and the library workspace."""
    return (12 * total_edges + 8 * (n_trees + 1) + 4 * total_edges + 4 * (total_edges + n_trees)
            + B.workspace_size(total_edges, max(n_trees, 1)))


class DendrogramServer:
    def __init__(self, hbm_budget_bytes: int, max_batch_edges: int = 32_000_000,
                 max_batch_trees: int = 4096, n_streams: int = 3, device="cuda",
                 clock=time.perf_counter, small_lane: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.budget = int(hbm_budget_bytes)
        self.max_batch_edges = int(max_batch_edges)
        self.max_batch_trees = int(max_batch_trees)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
        self.free_streams = deque(self.streams)
        self.pending: deque = deque()          # large lane
        self.pending_small: deque = deque()    # small lane
        self.inflight: List[_Batch] = []
        self.bytes_in_use = 0
        self.clock = clock
        self._next_bid = 0
        self.max_inflight = 0
        self.done: List[Result] = []
        B.load_library()
        self.small_cutoff = B.get_tuning()["small_max_edges"] if small_lane else -1

    # -- queue ---------------------------------------------------------------
    def submit(self, req: Request) -> None:
        if req.m > self.max_batch_edges or batch_footprint(req.m, 1) > self.budget:
            raise ValueError(f"request {req.rid} ({req.m} edges) can never fit the server")
        (self.pending_small if req.m <= self.small_cutoff else self.pending).append(req)

    def idle(self) -> bool:
        return not self.pending and not self.pending_small and not self.inflight

    # -- one scheduling round --------------------------------------------------
    def step(self) -> int:
        """Retire finished batches, admit new ones; returns batches admitted."""
        self.poll()
        admitted = 0
        while self.free_streams:
            lane = self._pick_lane()
            if lane is None:
                break
            reqs = self._take(lane)
            if not reqs:
                break
            self._launch(reqs)
            admitted += 1
        return admitted

    def _pick_lane(self):
        """The lane to admit from next: small requests first; a large batch
        never takes the last free stream while other batches run (a small
        request arriving meanwhile would wait behind it)."""
        if self.pending_small:
            return self.pending_small
        if self.pending and (len(self.free_streams) > 1 or not self.inflight
                             or self.small_cutoff < 0):
            return self.pending
        return None

    def _take(self, lane: deque) -> List[Request]:
        free = self.budget - self.bytes_in_use
        take: List[Request] = []
        m = 0
        while lane and len(take) < self.max_batch_trees:
            r = lane[0]
            if m + r.m > self.max_batch_edges:
                break
            if batch_footprint(m + r.m, len(take) + 1) > free:
                break
            take.append(lane.popleft())
            m += r.m
        return take

    def _launch(self, reqs: List[Request]) -> None:
        torch = self.torch
        stream = self.free_streams.popleft()
        t_admit = self.clock()
        offsets = [0]
        for r in reqs:
            offsets.append(offsets[-1] + r.m)
        m, t = offsets[-1], len(reqs)
        fp = batch_footprint(m, t)
        with torch.cuda.stream(stream):
            u = torch.cat([r.u for r in reqs]) if m else torch.empty(0, dtype=torch.int32,
                                                                     device=self.device)
            v = torch.cat([r.v for r in reqs]) if m else torch.empty_like(u)
            w = torch.cat([r.w for r in reqs]) if m else torch.empty(0, dtype=torch.float32,
                                                                     device=self.device)
            # offsets from pinned memory: an asynchronous copy that does not
            # wait for the stream (kept alive until the batch retires)
            off_h = torch.tensor(offsets, dtype=torch.int64).pin_memory()
            off = off_h.to(self.device, non_blocking=True)
            ws = torch.empty(B.workspace_size(m, max(t, 1)), dtype=torch.uint8, device=self.device)
            ep = torch.empty(m, dtype=torch.int32, device=self.device)
            vp = torch.empty(m + t, dtype=torch.int32, device=self.device)
            B.dendrogram_batched_planned(u, v, w, off, offsets, ws, (ep, vp))
            ev = torch.cuda.Event()
            ev.record(stream)
        self.bytes_in_use += fp
        self.inflight.append(_Batch(self._next_bid, reqs, stream, ev, ws, ep, vp, offsets, fp,
                                    t_admit, keep=[u, v, w, off, off_h]))
        self._next_bid += 1
        self.max_inflight = max(self.max_inflight, len(self.inflight))

    def poll(self) -> int:
        """Retire every finished batch; returns how many finished."""
        finished = 0
        still = []
        for b in self.inflight:
            if b.event.query():
                self._retire(b)
                finished += 1
            else:
                still.append(b)
        self.inflight = still
        return finished

    def _retire(self, b: _Batch) -> None:
        torch = self.torch
        t_done = self.clock()
        with torch.cuda.stream(b.stream):
            st = B.workspace_status(b.ws, raise_on_error=False)
        if st:
            raise B.PandoraError(st, f"batch {b.bid}")
        for k, r in enumerate(b.reqs):
            e0, e1 = b.offsets[k], b.offsets[k + 1]
            self.done.append(Result(r.rid, b.ep[e0:e1], b.vp[e0 + k:e1 + k + 1], r.t_arrival,
                                    b.t_admit, t_done, b.bid))
        self.bytes_in_use -= b.footprint
        self.free_streams.append(b.stream)

    def drain(self, poll_sleep: float = 20e-6) -> None:
        while not self.idle():
            if not self.step():
                time.sleep(poll_sleep)


def run_trace(server: DendrogramServer, requests: List[Request], arrivals: List[float],
              poll_sleep: float = 20e-6) -> List[Result]:
    """Feed requests at their arrival times (seconds from the start) and run
    the server until every request is done.  Returns results in finish order."""
    order = sorted(range(len(requests)), key=lambda i: arrivals[i])
    t0 = server.clock()
    k = 0
    while k < len(order) or not server.idle():
        now = server.clock() - t0
        while k < len(order) and arrivals[order[k]] <= now:
            r = requests[order[k]]
            r.t_arrival = t0 + arrivals[order[k]]
            server.submit(r)
            k += 1
        if not server.step() and server.inflight:
            time.sleep(poll_sleep)
    return server.done
