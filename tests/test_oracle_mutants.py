"""The pins of the dendrogram oracle catch plausible mistakes.

Each case plants one mistake in a copy of oracle/kruskal.c, compiles the copy
with gcc into a temporary library (CPU only) and runs the independent routes
of tests/pins.py (brute force from the definition, the top-down
construction) on random small trees with ties and special floats, plus the
hand-worked fixtures under tests/golden/.  Every mutant must fail at least
one of them; the unmutated copy must pass them all.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import golden_io
import pins
from paper_2401_06089_gb300 import inputs

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "kruskal.c")

MUTANTS = {
    "larger index first on ties": ("    return a < b;\n}", "    return a > b;\n}"),
    "positive zero first": ("        return sa; /* the negative zero is the lighter one */",
                            "        return sb;"),
    "sorted heaviest first": ("        if (lighter(w, idx[j], idx[i]))",
                              "        if (lighter(w, idx[i], idx[j]))"),
    "one top node left without parent": ("        for (int s = 0; s < 2; ++s) {",
                                         "        for (int s = 0; s < 1; ++s) {"),
    "root is the lightest edge": ("    edge_parent[order[n_edges - 1]] = -1;",
                                  "    edge_parent[order[0]] = -1;"),
    "new top on the absorbed root": ("        top[a] = ~e;", "        top[b] = ~e;"),
    "union links the wrong way": ("        uf[b] = a;\n        size[a] += size[b];",
                                  "        uf[a] = b;\n        size[a] += size[b];"),
}


def _build(tmp_path, name, text):
    src = tmp_path / f"{name}.c"
    lib = tmp_path / f"{name}.so"
    src.write_text(text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-pthread", "-o", str(lib),
                    str(src), "-lm", "-lpthread"], check=True)
    so = ctypes.CDLL(str(lib))
    so.oracle_dendrogram.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int64] + \
        [ctypes.c_void_p] * 2
    so.oracle_dendrogram.restype = ctypes.c_int

    def dendrogram(u, v, w):
        u = np.ascontiguousarray(u, np.int32)
        v = np.ascontiguousarray(v, np.int32)
        w = np.ascontiguousarray(w, np.float32)
        m = len(w)
        ep = np.full(max(m, 1), -7, np.int32)
        vp = np.full(m + 1, -7, np.int32)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)   # noqa: E731
        st = so.oracle_dendrogram(p(u), p(v), p(w), m, p(ep), p(vp))
        return st, ep[:m], vp
    return dendrogram


def _pins_hold(dendrogram):
    rng = np.random.default_rng(77)
    specials = np.array([-np.inf, -1.5, -0.0, 0.0, 1e-45, 1.0, np.inf], np.float32)
    for k in range(120):
        n = int(rng.integers(2, 30))
        t = inputs.rrt(n, int(rng.integers(1 << 30)))
        if k % 3 == 1:
            t = inputs.with_weights(t, rng.integers(0, 3, size=n - 1).astype(np.float32))
        elif k % 3 == 2:
            t = inputs.with_weights(t, rng.choice(specials, size=n - 1))
        st, ep, vp = dendrogram(t.u, t.v, t.w)
        if st != 0:
            return False
        bep, bvp = pins.brute_force(t.u, t.v, t.w)
        if not (np.array_equal(ep, bep) and np.array_equal(vp, bvp)):
            return False
        tep, tvp = pins.top_down(t.u, t.v, t.w)
        if not (np.array_equal(ep, tep) and np.array_equal(vp, tvp)):
            return False
    for path in golden_io.all_cases():
        u, v, w, gep, gvp = golden_io.load(path)
        st, ep, vp = dendrogram(u, v, w)
        if st != 0 or not (np.array_equal(ep, gep) and np.array_equal(vp, gvp)):
            return False
    return True


def test_unmutated_copy_passes(tmp_path):
    assert _pins_hold(_build(tmp_path, "kruskal_copy", open(SRC).read()))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    text = open(SRC).read()
    old, new = MUTANTS[name]
    assert text.count(old) == 1, old
    assert not _pins_hold(_build(tmp_path, "kruskal_mutant", text.replace(old, new))), name
