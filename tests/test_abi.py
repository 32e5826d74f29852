"""The C-ABI library builds, loads without a GPU and exports what include/ declares.

CPU only: no kernel is launched (only host-side entry points are called).
"""
import ctypes
import glob
import os
import re

import pytest

from paper_2401_06089_gb300 import build as libbuild
from paper_2401_06089_gb300 import _binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(pandora_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return ctypes.CDLL(libbuild.LIB)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("pandora_dendrogram", "pandora_dendrogram_batched", "pandora_workspace_size",
                 "pandora_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    bl = _binding.load_library()
    assert bl.pandora_version() >= 100
    for code, name in _binding.STATUS_NAMES.items():
        assert _binding.status_string(code)
    assert _binding.workspace_size(0, 1) > 0
    a = _binding.workspace_size(1000, 1)
    b = _binding.workspace_size(2000, 1)
    assert b > a
    with pytest.raises(_binding.PandoraError):
        _binding.workspace_size(-1, 1)


def test_argument_errors_are_reported_before_any_launch(lib):
    bl = _binding.load_library()
    null = ctypes.c_void_p(0)
    # negative size, null outputs: rejected on the host, nothing enqueued
    assert bl.pandora_dendrogram(null, null, null, -1, null, null, null) == 1
    assert bl.pandora_dendrogram(null, null, null, 5, null, null, null) == 1
    assert bl.pandora_dendrogram(null, null, null, 2**31, null, null, null) == 1
    assert bl.pandora_dendrogram_batched(null, null, null, null, 3, 10, null, null, null) == 1
    sz = ctypes.c_size_t(0)
    assert bl.pandora_workspace_size(10, 0, ctypes.byref(sz)) == 1
    # flat clusters: min_cluster_size below 2, negative size, null arrays,
    # above the size limit
    nc = ctypes.c_int64(-5)
    flat = bl.pandora_hdbscan_labels
    assert flat(null, null, null, 10, 1, null, null, ctypes.byref(nc), null) == 1
    assert flat(null, null, null, -1, 2, null, null, ctypes.byref(nc), null) == 1
    assert flat(null, null, null, 10, 2, null, null, ctypes.byref(nc), null) == 1
    assert flat(null, null, null, _binding.FLAT_MAX_VERTICES + 1, 2, null, null,
                ctypes.byref(nc), null) == 10
    assert nc.value == -5


def test_noalloc_scratch_holds_the_largest_accepted_input():
    """pandora_dendrogram_noalloc's static scratch (32 MiB) must hold the
    workspace of its largest accepted input, PANDORA_NOALLOC_MAX_EDGES."""
    text = open(os.path.join(ROOT, "include", "pandora.h")).read()
    max_edges = int(re.search(r"#define PANDORA_NOALLOC_MAX_EDGES (\d+)", text).group(1))
    assert _binding.workspace_size(max_edges, 1) <= 32 << 20


def test_tuning_round_trip_and_validation(lib):
    """Small-tree settings: defaults, a valid change, rejected changes (host only)."""
    saved = _binding.get_tuning()
    try:
        assert 0 <= saved["small_max_edges"] <= _binding.SMALL_CAP
        assert len(saved["small_threads"]) == _binding.SMALL_BUCKETS
        thr = [256, 512, 1024] * 4 + [256]
        got = _binding.set_tuning(1234, thr, 75)
        assert got == {"small_max_edges": 1234, "small_threads": thr, "split_min_permille": 75}
        assert _binding.set_tuning(10**6)["small_max_edges"] == _binding.SMALL_CAP   # clamped
        for bad_thr in ([128] * 13, [512] * 12 + [300]):
            with pytest.raises(_binding.PandoraError) as ei:
                _binding.set_tuning(100, bad_thr)
            assert ei.value.code == 1
        with pytest.raises(_binding.PandoraError):
            _binding.set_tuning(-1)
        for bad_permille in (-1, 1001):
            with pytest.raises(_binding.PandoraError):
                _binding.set_tuning(100, None, bad_permille)
        assert _binding.get_tuning()["small_max_edges"] == _binding.SMALL_CAP   # unchanged
        assert lib.pandora_set_tuning(None) == 1
        assert lib.pandora_get_tuning(None) == 1
    finally:
        _binding.set_tuning(saved["small_max_edges"], saved["small_threads"],
                            saved["split_min_permille"])


def test_batched_workspace_holds_the_packed_forest():
    """A batched call's workspace also holds the large trees packed as one forest."""
    single = _binding.workspace_size(100_000, 1)
    batched = _binding.workspace_size(100_000, 50)
    assert batched >= single + 5 * 4 * 100_000


def test_planned_host_offsets_checked_before_any_launch(lib):
    """The planned batched call rejects host offsets that are not a partition
    of [0, total_edges), and a missing workspace, before enqueuing anything."""
    bl = _binding.load_library()
    null = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(256)   # never dereferenced: the call returns first
    bad = (ctypes.c_int64 * 4)(0, 5, 3, 10)
    short = (ctypes.c_int64 * 4)(0, 5, 7, 9)
    good = (ctypes.c_int64 * 4)(0, 5, 7, 10)
    args = (fake, fake, fake, fake)
    for h in (bad, short):
        assert bl.pandora_dendrogram_batched_planned(*args, h, 3, 10, fake, fake, null, 0,
                                                      null) == 1
    assert bl.pandora_dendrogram_batched_planned(*args, null, 3, 10, fake, fake, null, 0,
                                                  null) == 1
    assert bl.pandora_dendrogram_batched_planned(*args, good, 3, 10, fake, fake, null, 0,
                                                  null) == 9


def test_sort_pairs_workspace_follows_the_digit_plan(lib):
    """pandora_sort_pairs_workspace_size is host-only.  Keys of 25 to 27 bits
    take three passes of 9-bit digits, whose look-back table has 512 entries
    per 4096-key tile against 256 for the 8-bit plans (up to 24 and from 28
    bits): the workspace grows by exactly that table.  Bad arguments are
    rejected before any launch."""
    bl = _binding.load_library()
    sz = ctypes.c_size_t(0)

    def ws(n, bits):
        assert bl.pandora_sort_pairs_workspace_size(n, bits, ctypes.byref(sz)) == 0
        return sz.value

    n = 4096 * 1000
    tiles = 1000
    base = ws(n, 24)
    assert ws(n, 28) == base == ws(n, 32) == ws(n, 8)
    for bits in (25, 26, 27):
        assert ws(n, bits) == base + tiles * (512 - 256) * 8
    assert ws(2 * n, 24) > base
    null = ctypes.c_void_p(0)
    for args in ((-1, 24), (10, 0), (10, 33)):
        assert bl.pandora_sort_pairs_workspace_size(*args, ctypes.byref(sz)) == 1
    assert bl.pandora_sort_pairs_workspace_size(10, 24, ctypes.POINTER(ctypes.c_size_t)()) == 1
    # the sort itself: bad sizes and null arrays are rejected on the host
    sort = bl.pandora_sort_pairs
    assert sort(null, null, -1, 24, null, null, null, 0, null) == 1
    assert sort(null, null, 10, 24, null, null, null, 0, null) == 1
    assert sort(null, null, 10, 40, null, null, null, 0, null) == 1
    assert sort(null, null, 0, 24, null, null, null, 0, null) == 0
