"""Sharding of a batch across ranks: host logic, and a world-size-2 run over
gloo on CPU (each rank solves its shard with the oracle; rank 0 gathers and
checks the reassembled batch against the oracle on the whole batch)."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2401_06089_gb300 import inputs
from paper_2401_06089_gb300.sharding import merge_outputs, shard_trees, sub_batch


def test_every_tree_on_exactly_one_rank_and_balanced():
    rng = np.random.default_rng(0)
    m = inputs.log_uniform_sizes(rng, 4096, 100, 1_000_000) - 1
    for world in (1, 2, 3, 8):
        shards = shard_trees(m, world)
        allt = np.concatenate(shards)
        assert sorted(allt.tolist()) == list(range(len(m)))
        loads = [int(m[s].sum()) for s in shards]
        # LPT bound: max load <= mean + largest tree
        assert max(loads) <= m.sum() / world + m.max()
        for s in shards:
            assert np.all(np.diff(s) > 0)


def test_more_ranks_than_trees():
    shards = shard_trees([5, 3], 4)
    assert sorted(np.concatenate(shards).tolist()) == [0, 1]
    assert sum(len(s) == 0 for s in shards) == 2


def test_sub_batch_and_merge_roundtrip():
    b = inputs.batch(30, 1, 500, seed=3)
    oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
    m = np.diff(b.edge_offsets)
    shards = shard_trees(m, 3)
    outs = []
    for s in shards:
        u, v, w, off = sub_batch(b.u, b.v, b.w, b.edge_offsets, s)
        outs.append(oracle.dendrogram_batched(u, v, w, off))
    ep, vp = merge_outputs(b.edge_offsets, shards, outs)
    np.testing.assert_array_equal(ep, oep)
    np.testing.assert_array_equal(vp, ovp)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = inputs.batch(40, 1, 2000, seed=9)
    m = np.diff(b.edge_offsets)
    shards = shard_trees(m, world)
    u, v, w, off = sub_batch(b.u, b.v, b.w, b.edge_offsets, shards[rank])
    mine = oracle.dendrogram_batched(u, v, w, off)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, mine))
    if rank == 0:
        outs = [o for _, o in sorted(gathered, key=lambda x: x[0])]
        ep, vp = merge_outputs(b.edge_offsets, shards, outs)
        oep, ovp = oracle.dendrogram_batched(b.u, b.v, b.w, b.edge_offsets)
        ok = np.array_equal(ep, oep) and np.array_equal(vp, ovp)
        with open(result_path, "w") as f:
            f.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_over_gloo(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    result = tmp_path / "result.txt"
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(result))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert result.read_text() == "ok"
