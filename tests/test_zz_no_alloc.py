"""The allocation-free entry point, pandora_dendrogram_noalloc.

Some callers cannot allocate device memory when they need a dendrogram: all
of their GPU memory is owned by another allocator (a framework that reserved
the device up front), or they run a latency-critical loop in which
cudaMalloc/cudaFree would synchronise the device.  For them the library has
one entry point whose scratch is a fixed array in its device image.  These
tests call it through the C ABI and require the same outputs as
pandora_dendrogram and as the CPU oracle (exact equality: the outputs are
integers) on two calls in a row, the second smaller than the first so that
contents left behind by the first call cannot leak into the second, and they
check in a fresh process that the calls leave the device's free memory
unchanged (nothing is allocated, not even from the library's pool).

The file name makes pytest collect it last: should it fail, a run that stops
at the first failure (-x) has already run every other test.
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2401_06089_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_EDGES = 262143          # PANDORA_NOALLOC_MAX_EDGES in include/pandora.h
SIZE_LIMIT = 10             # PANDORA_ERR_SIZE_LIMIT


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_06089_gb300 as pd
    lib = pd.load_library()
    P = ctypes.c_void_p
    lib.pandora_dendrogram_noalloc.argtypes = [P, P, P, ctypes.c_int64, P, P, P]
    lib.pandora_dendrogram_noalloc.restype = ctypes.c_int
    return lib


def _noalloc(lib, t):
    dev = torch.device("cuda")
    u = torch.from_numpy(t.u).to(dev)
    v = torch.from_numpy(t.v).to(dev)
    w = torch.from_numpy(t.w).to(dev)
    ep = torch.full((t.m,), -7, dtype=torch.int32, device=dev)
    vp = torch.full((t.m + 1,), -7, dtype=torch.int32, device=dev)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.pandora_dendrogram_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                        ctypes.c_void_p(w.data_ptr()), t.m,
                                        ctypes.c_void_p(ep.data_ptr()),
                                        ctypes.c_void_p(vp.data_ptr()), stream)
    assert st == 0, st
    return u, v, w, ep.cpu().numpy(), vp.cpu().numpy()


def test_noalloc_matches_pandora_dendrogram_on_two_calls(lib):
    import paper_2401_06089_gb300 as pd
    for t in (inputs.rrt(MAX_EDGES + 1, seed=21), inputs.path_skewed(5000, seed=22)):
        u, v, w, ep, vp = _noalloc(lib, t)
        rep, rvp = pd.dendrogram(u, v, w)
        np.testing.assert_array_equal(ep, rep.cpu().numpy())
        np.testing.assert_array_equal(vp, rvp.cpu().numpy())
        oep, ovp = oracle.dendrogram(t.u, t.v, t.w)
        np.testing.assert_array_equal(ep, oep)
        np.testing.assert_array_equal(vp, ovp)


_FRESH = r"""
import ctypes, json, sys
sys.path.insert(0, sys.argv[1])
import torch
import paper_2401_06089_gb300 as pd
from paper_2401_06089_gb300 import inputs
lib = pd.load_library()
P = ctypes.c_void_p
lib.pandora_dendrogram_noalloc.argtypes = [P, P, P, ctypes.c_int64, P, P, P]
dev = torch.device("cuda")
trees = [inputs.rrt(200000, 31), inputs.rrt(3000, 32)]
bufs = []
for t in trees:
    bufs.append([torch.from_numpy(t.u).to(dev), torch.from_numpy(t.v).to(dev),
                 torch.from_numpy(t.w).to(dev), torch.empty(t.m, dtype=torch.int32, device=dev),
                 torch.empty(t.m + 1, dtype=torch.int32, device=dev)])
# load the library's kernels and start its runtime through a call that takes
# a caller workspace (no allocation either)
t = trees[1]
b = bufs[1]
ws = torch.empty(pd.workspace_size(t.m), dtype=torch.uint8, device=dev)
pd.dendrogram_async(b[0], b[1], b[2], ws, (b[3], b[4]))
torch.cuda.synchronize()
stream = P(torch.cuda.current_stream().cuda_stream)
free = [torch.cuda.mem_get_info()[0]]
for t, b in zip(trees, bufs):
    st = lib.pandora_dendrogram_noalloc(*[P(x.data_ptr()) for x in b[:3]], t.m,
                                        P(b[3].data_ptr()), P(b[4].data_ptr()), stream)
    torch.cuda.synchronize()
    free.append(torch.cuda.mem_get_info()[0])
    assert st == 0, st
print(json.dumps({"free": free}))
"""


def test_noalloc_allocates_nothing_in_a_fresh_process(lib):
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    r = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True,
                       timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    free = json.loads(r.stdout.strip().splitlines()[-1])["free"]
    assert free[0] == free[1] == free[2], free


def test_noalloc_rejects_inputs_above_the_limit(lib):
    dev = torch.device("cuda")
    small = torch.zeros(4, dtype=torch.int32, device=dev)
    wsmall = torch.zeros(4, dtype=torch.float32, device=dev)
    p = lambda x: ctypes.c_void_p(x.data_ptr())
    st = lib.pandora_dendrogram_noalloc(p(small), p(small), p(wsmall), MAX_EDGES + 1, p(small),
                                        p(small), ctypes.c_void_p(0))
    assert st == SIZE_LIMIT
