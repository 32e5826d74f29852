"""The autotuner's decisions from measured timings (host logic, no GPU): the
block size per bucket, the cutoff, and the split threshold; and the shipped
tuning file is a valid setting."""
import json
import os

import pytest

from paper_2401_06089_gb300 import autotune, _binding


def _row(k, solver, pipeline, best=256, edges=1_000_000):
    return {"bucket": k, "best_threads": best, "solver_ms": {str(best): solver},
            "pipeline_ms": pipeline, "solver_ns_per_edge": 1e6 * solver / edges,
            "pipeline_ns_per_edge": 1e6 * pipeline / edges}


def test_cutoff_is_top_of_last_winning_bucket_from_zero():
    rows = [_row(k, 1.0, 2.0) for k in range(8)] + [_row(8, 3.0, 2.0)] + \
        [_row(k, 1.0, 2.0) for k in range(9, 13)]
    threads, cutoff = autotune.choose_threads_and_cutoff(rows)
    assert cutoff == (1 << 8) - 1          # bucket 8 loses: stop below it
    assert threads == [256] * 13
    rows = [_row(k, 1.0, 2.0, best=1024 if k > 9 else 256) for k in range(13)]
    threads, cutoff = autotune.choose_threads_and_cutoff(rows)
    assert cutoff == _binding.SMALL_CAP
    assert threads[-1] == 1024 and threads[0] == 256
    rows = [_row(0, 3.0, 2.0)] + [_row(k, 1.0, 2.0) for k in range(1, 13)]
    assert autotune.choose_threads_and_cutoff(rows)[1] == 0


def test_split_threshold_is_break_even_share():
    # saving 0.4 ns per small edge, packing 0.1 ns per large edge:
    # s * 0.4 = (1 - s) * 0.1  ->  s = 0.2  ->  200 per mille
    rows = [_row(k, 1.0, 1.4, edges=1_000_000) for k in range(13)]
    saving, permille = autotune.choose_split_permille(rows, 4096, 0.1)
    assert saving == pytest.approx(0.4)
    assert permille == 200
    # no saving: never split a mixed batch
    rows = [_row(k, 2.0, 1.0) for k in range(13)]
    assert autotune.choose_split_permille(rows, 4096, 0.1)[1] == 1000


def test_shipped_tuning_file_is_a_valid_setting():
    path = os.path.join(os.path.dirname(_binding.__file__), "tuning_gb300.json")
    cfg = json.load(open(path))
    assert 0 <= cfg["small_max_edges"] <= _binding.SMALL_CAP
    assert len(cfg["small_threads"]) == _binding.SMALL_BUCKETS
    assert all(t in (256, 512, 1024) for t in cfg["small_threads"])
    assert 0 <= cfg["split_min_permille"] <= 1000
    saved = _binding.get_tuning()
    try:
        got = _binding.load_tuning(path)
        assert got["small_max_edges"] == cfg["small_max_edges"]
    finally:
        _binding.set_tuning(saved["small_max_edges"], saved["small_threads"],
                            saved["split_min_permille"])
