"""The pins of the float32 reading of the EMST oracle catch plausible
mistakes: each case plants one in a copy of oracle/emst.py (in memory, on the
CPU) and runs tests/test_emst_f32_oracle.py's pins against the copy."""
import os
import types

import pytest

import test_emst_f32_oracle as P

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "emst.py")

MUTANTS = {
    "ties by the larger id first": ("order = np.lexsort((bhi[out], blo[out], bw[out]))",
                                    "order = np.lexsort((blo[out], bhi[out], bw[out]))"),
    "ties ignored when updating": (
        "better = (w2 < bw) | ((w2 == bw) & ((lo < blo) | ((lo == blo) & (hi < bhi))))",
        "better = (w2 < bw)"),
    "core skips the point itself": ("core2[a] = np.partition(d2, min_pts - 1)[min_pts - 1]",
                                    "core2[a] = np.partition(d2, min_pts)[min_pts]"),
    "distances in float64": ("        dk = p[:, k] - p[a, k]                     # float32 subtraction",
                             "        dk = p[:, k].astype(np.float64) - float(p[a, k])"),
    "one core distance": ("w2 = np.maximum(np.maximum(core2, core2[x]), d2)",
                          "w2 = np.maximum(core2, d2)"),
}


def _load(mutation):
    text = open(SRC).read()
    old, new = mutation
    assert text.count(old) == 1, old
    mod = types.ModuleType("emst_f32_mutant")
    exec(compile(text.replace(old, new), "emst_f32_mutant", "exec"), mod.__dict__)
    return mod


def _pins_hold(mod, monkeypatch):
    monkeypatch.setattr(P, "emst", mod)
    try:
        for seed in range(8):
            P.test_integer_coordinates_match_float64_oracle(seed)
        for seed in range(6):
            P.test_weights_and_core_distances_by_scalars(seed)
        for n in (2, 3, 4, 5, 6):
            P.test_minimum_over_all_spanning_trees(n)
        for seed in range(16):
            P.test_cut_property_under_the_total_order(seed)
    except (AssertionError, ValueError, IndexError):
        return False
    return True


def test_unmutated_copy_passes(monkeypatch):
    assert _pins_hold(_load(("def mr_emst_f32", "def mr_emst_f32")), monkeypatch)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(monkeypatch, name):
    assert not _pins_hold(_load(MUTANTS[name]), monkeypatch), name
