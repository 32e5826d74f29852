"""The benchmark's reference arm runs on the CPU: its JSON line carries the
keys the benchmark contract asks for; and the benchmark's host-side helpers."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["unit"] == "edges/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == (os.cpu_count() or 1)
    # the line names the sample it timed, not the full-size workload
    assert d["config"]["workload"] == "rrt_1e8_sample_n10000000"
    assert d["config"]["n_edges"] == 10_000_000 - 1
    assert d["config"]["sample_of"].startswith("rrt_1e8")


def test_structure_check_accepts_dendrograms_and_rejects_corruptions():
    """bench.py --check validates outputs without the oracle; the checks must
    hold on correct dendrograms (from the oracle here, on the CPU) and fail
    on each kind of corruption."""
    import importlib.util

    import numpy as np

    import oracle
    from paper_2401_06089_gb300 import inputs

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    check = bench.dendrogram_structure
    for seed in range(6):
        t = inputs.rrt(3000, seed) if seed % 2 else inputs.path(3000, seed, kind="random")
        w = t.w if seed < 4 else np.where(np.arange(t.m) % 2, 0.0, -0.0).astype(np.float32)
        ep, vp = oracle.dendrogram(t.u, t.v, w)
        assert check(t.u, t.v, w, ep, vp)["ok"]
        e = int(np.flatnonzero(ep >= 0)[seed])
        bad = ep.copy()
        bad[e] = -1                                  # two roots
        assert not check(t.u, t.v, w, bad, vp)["ok"]
        bad = ep.copy()
        bad[ep[e]] = e                               # a parent earlier than its child
        assert not check(t.u, t.v, w, bad, vp)["ok"]
        badv = vp.copy()
        x = int(np.flatnonzero(vp != vp[0])[0])
        badv[x] = vp[0]                              # three children / not the lightest
        assert not check(t.u, t.v, w, ep, badv)["ok"]
    one = check(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32),
                np.zeros(0, np.int32), np.full(1, -1, np.int32))
    assert one["ok"]


def test_dendrogram_height_and_skewness():
    """The skewness the bench reports (Section 3.1: height over log2 n) on
    dendrograms whose height is known: a chain and a balanced tree."""
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    # a chain: e0 -> e1 -> e2 -> e3 (root); vertices 0, 1 under e0, then one
    # vertex under each further edge: the deepest vertex is 4 edges down
    ep = torch.tensor([1, 2, 3, -1])
    vp = torch.tensor([0, 0, 1, 2, 3])
    assert bench.dendrogram_height(ep, vp) == 4
    # balanced: root e1 over e0 and e2, two vertices under each
    ep = torch.tensor([1, -1, 1])
    vp = torch.tensor([0, 0, 2, 2])
    assert bench.skewness(ep, vp) == {"height": 2, "ideal_log2_n": 2.0, "ratio": 1.0}
    # a long chain, deeper than a single pointer-jumping step
    m = 1000
    ep = torch.arange(1, m + 1)
    ep[-1] = -1
    vp = torch.cat([torch.tensor([0]), torch.arange(m)])
    assert bench.dendrogram_height(ep, vp) == m
