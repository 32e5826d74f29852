"""The pins of the flat-cluster oracle catch plausible mistakes.

Each case plants one mistake in a copy of oracle/flat.py's source (on the
CPU, in memory) and runs the pins of tests/test_flat_oracle.py against the
copy: the component sweep, the exhaustive selection search, the labels from
the member lists and the hand-worked trees.  Every mutant must fail at least
one of them.
"""
import os
import types

import numpy as np
import pytest

import oracle
import test_flat_oracle as P
from paper_2401_06089_gb300 import inputs

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "flat.py")

MUTANTS = {
    "child wins a tie": ('if Fraction(C["stability"]) >= tot:',
                         'if Fraction(C["stability"]) > tot:'),
    "root is a candidate": ("for ci in range(len(clusters) - 1, 0, -1):",
                            "for ci in range(len(clusters) - 1, -1, -1):"),
    # (a split on one large side would descend into vertices and never end)
    "never split": ("if big1 and big2:", "if big1 and big2 and False:"),
    "child born at lambda 0": ('clusters.append({"edge": c, "parent": ci, "birth": lam[e],',
                               'clusters.append({"edge": c, "parent": ci, "birth": 0.0,'),
    "child term without its size": ('total += D["size"] * Fraction(D["birth"] - C["birth"])',
                                    'total += Fraction(D["birth"] - C["birth"])'),
    "leaving term sign": ('total += Fraction(lx - C["birth"])',
                          'total += Fraction(C["birth"] - lx)'),
    "child totals dropped": ('total += D["size"] * Fraction(D["birth"] - C["birth"])',
                             'pass'),
    "strict size threshold": ("big1 = csize(k1, c1) >= mcs\n        big2 = csize(k2, c2) >= mcs",
                              "big1 = csize(k1, c1) > mcs\n        big2 = csize(k2, c2) > mcs"),
    "descendants kept": ("                selected[d] = False\n", "                pass\n"),
    "numbered by creation order": ("sorted(firsts, key=lambda c: firsts[c])", "sorted(firsts)"),
    "weights not inverted": ("lam = [1.0 / float(x) for x in wd]", "lam = [float(x) for x in wd]"),
}


def _load(mutation):
    text = open(SRC).read()
    old, new = mutation
    assert text.count(old) == 1, old
    mod = types.ModuleType("flat_mutant")
    exec(compile(text.replace(old, new), "flat_mutant", "exec"), mod.__dict__)
    return mod


def _pins_hold(mod):
    """True when every pin passes for this copy of the oracle."""
    try:
        for seed in range(24):
            rng = np.random.default_rng(seed)
            n = int(rng.integers(2, 24))
            t = inputs.rrt(n, seed) if seed % 2 else inputs.path(max(n, 2), seed, kind="random")
            w = t.w
            if seed % 4 == 0:
                w = rng.integers(1, 4, size=t.m).astype(np.float32)
            elif seed % 4 == 2:
                w = np.exp2(rng.uniform(-60, 60, size=t.m)).astype(np.float32)
            mcs = int(rng.integers(2, 6))
            ep, vp = oracle.dendrogram(t.u, t.v, w)
            labels, info = mod.hdbscan_labels(ep, vp, w, mcs, members=True)
            ref = P.sweep_clusters(t.u, t.v, w, mcs)
            got = sorted((tuple(C["members"]), C["birth"], C["stability"])
                         for C in info["clusters"])
            exp = sorted((tuple(sorted(p)), b, s) for p, b, s, _ in ref)
            assert got == exp
            P.check_selection(info)
            np.testing.assert_array_equal(labels, P.labels_from(info, t.n))
        # the hand-worked trees of the pins
        u = np.array([1, 2, 3, 4, 5, 6], np.int32)
        v = np.array([0, 0, 2, 1, 3, 4], np.int32)
        w = np.array([1, 2, 0.25, 1, 0.25, 0.5], np.float32)
        ep, vp = oracle.dendrogram(u, v, w)
        labels, _ = mod.hdbscan_labels(ep, vp, w, 2)
        np.testing.assert_array_equal(labels, [0, 0, 1, 1, 0, 1, 0])
        u = np.array([0, 1, 2, 4, 5, 6, 3, 0], np.int32)
        v = np.array([1, 2, 3, 5, 6, 7, 4, 8], np.int32)
        w = np.array([1, 1, 1, 1, 1, 1, 10, 100], np.float32)
        ep, vp = oracle.dendrogram(u, v, w)
        labels, info = mod.hdbscan_labels(ep, vp, w, 3)
        np.testing.assert_array_equal(labels, [0, 0, 0, 0, 1, 1, 1, 1, -1])
        assert [C["stability"] for C in info["clusters"][1:]] == [4 * (1.0 - 0.1)] * 2
    except (AssertionError, ValueError, IndexError, KeyError):
        return False
    return True


def test_unmutated_copy_passes():
    text = open(SRC).read()
    mod = types.ModuleType("flat_copy")
    exec(compile(text, "flat_copy", "exec"), mod.__dict__)
    assert _pins_hold(mod)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name):
    assert not _pins_hold(_load(MUTANTS[name])), name
