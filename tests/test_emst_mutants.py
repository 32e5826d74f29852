"""The pins of the mutual-reachability MST oracle catch plausible mistakes:
each case plants one in a copy of oracle/emst.py (in memory, on the CPU) and
runs the pins of tests/test_emst_oracle.py against the copy."""
import os
import types

import numpy as np
import pytest

import test_emst_oracle as P

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "emst.py")

MUTANTS = {
    "core skips the point itself": ("core[a] = np.sort(d)[min_pts - 1]",
                                    "core[a] = np.sort(d)[min(min_pts, n - 1)]"),
    "core of one endpoint only": ("mr = np.maximum(np.maximum(core, core[x]), d)",
                                  "mr = np.maximum(core, d)"),
    "plain distance": ("mr = np.maximum(np.maximum(core, core[x]), d)", "mr = d"),
    "squared distance": ('d = np.sqrt(np.einsum("ij,ij->i", diff, diff))\n        mr',
                         'd = np.einsum("ij,ij->i", diff, diff)\n        mr'),
    "keeps the first candidate": ("upd = (~in_tree) & (mr < best)",
                                  "upd = (~in_tree) & (best == np.inf)"),
}


def _load(mutation):
    text = open(SRC).read()
    old, new = mutation
    assert text.count(old) == 1, old
    mod = types.ModuleType("emst_mutant")
    exec(compile(text.replace(old, new), "emst_mutant", "exec"), mod.__dict__)
    return mod


def _pins_hold(mod, monkeypatch):
    monkeypatch.setattr(P, "emst", mod)
    try:
        for seed in range(8):
            P.test_core_distances_exact_ranking(seed)
        for seed in range(10):
            P.test_weights_match_scipy(seed)
        for n in (2, 3, 4, 5, 6):
            P.test_minimum_over_all_spanning_trees(n)
        P.test_line_closed_form()
        for seed in range(4):
            P.test_cut_property(seed)
    except (AssertionError, ValueError, IndexError):
        return False
    return True


def test_unmutated_copy_passes(monkeypatch):
    pytest.importorskip("scipy")
    mod = types.ModuleType("emst_copy")
    exec(compile(open(SRC).read(), "emst_copy", "exec"), mod.__dict__)
    assert _pins_hold(mod, monkeypatch)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    pytest.importorskip("scipy")
    assert not _pins_hold(_load(MUTANTS[name]), monkeypatch), name
