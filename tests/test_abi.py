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


def test_noalloc_scratch_holds_the_largest_accepted_input():
    """pandora_dendrogram_noalloc's static scratch (32 MiB) must hold the
    workspace of its largest accepted input, PANDORA_NOALLOC_MAX_EDGES."""
    text = open(os.path.join(ROOT, "include", "pandora.h")).read()
    max_edges = int(re.search(r"#define PANDORA_NOALLOC_MAX_EDGES (\d+)", text).group(1))
    assert _binding.workspace_size(max_edges, 1) <= 32 << 20
