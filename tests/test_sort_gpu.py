"""The library's stable radix sort of (key, value) pairs on its own
(``pandora_sort_pairs``), for every digit plan it uses.

The dendrogram sorts the edges by weight (ties by index, Section 3.1) and
again by chain key, ties in rank order (Section 3.3.3); both are this sort.
Its result has a plain definition: the pairs ordered by key, equal keys in
input order, which numpy's stable argsort computes.  The checks are exact
(integers), at sizes that span many 4096-key tiles and end in a ragged tail,
for key widths that select each plan: three passes of 9 and 8 or 9 bits
from 25 to 27 bits (the chain keys of 8.4 to 67 million edges), 8-bit
digits otherwise.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_06089_gb300 as pd
    pd.load_library()
    return pd


def _check(pd, keys, key_bits):
    vals = np.arange(len(keys), dtype=np.uint32) * np.uint32(2654435761)
    dev = torch.device("cuda")
    tk = torch.from_numpy(keys.view(np.int32)).to(dev)
    tv = torch.from_numpy(vals.view(np.int32)).to(dev)
    ko, vo = pd.sort_pairs(tk, tv, key_bits)
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), vals[order])


BITS = [1, 8, 13, 16, 24, 25, 26, 27, 28, 29, 30, 31, 32]


@pytest.mark.parametrize("key_bits", BITS)
def test_uniform_keys_every_plan(pd, key_bits):
    rng = np.random.default_rng(key_bits)
    n = 4096 * 37 + 1111
    keys = rng.integers(0, 1 << key_bits, n, dtype=np.uint64).astype(np.uint32)
    _check(pd, keys, key_bits)


@pytest.mark.parametrize("key_bits", [24, 25, 27, 28, 32])
def test_heavy_duplicates_keep_input_order(pd, key_bits):
    # few distinct keys, spread over every digit of the plan: long runs of
    # equal keys across many tiles, where only stability decides the order
    rng = np.random.default_rng(100 + key_bits)
    distinct = rng.integers(0, 1 << key_bits, 7, dtype=np.uint64).astype(np.uint32)
    keys = distinct[rng.integers(0, 7, 4096 * 23 + 77)]
    _check(pd, keys, key_bits)


@pytest.mark.parametrize("key_bits", [26, 28])
def test_skewed_digits(pd, key_bits):
    # one key value holds most of the input (a root chain), the rest uniform
    rng = np.random.default_rng(7)
    n = 200_003
    keys = rng.integers(0, 1 << key_bits, n, dtype=np.uint64).astype(np.uint32)
    keys[rng.random(n) < 0.8] = np.uint32((1 << key_bits) - 1)
    _check(pd, keys, key_bits)


@pytest.mark.parametrize("n", [1, 2, 4095, 4096, 4097])
def test_small_and_tile_edges(pd, n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 1 << 28, n, dtype=np.uint64).astype(np.uint32)
    _check(pd, keys, 28)


@pytest.mark.parametrize("key_bits", [27, 28])
def test_large_input(pd, key_bits):
    rng = np.random.default_rng(11)
    n = 3_000_001
    keys = rng.integers(0, 1 << key_bits, n, dtype=np.uint64).astype(np.uint32)
    _check(pd, keys, key_bits)


def test_empty_and_key_above_bits(pd):
    dev = torch.device("cuda")
    e = torch.empty(0, dtype=torch.int32, device=dev)
    ko, vo = pd.sort_pairs(e, e, 28)
    assert ko.numel() == 0 and vo.numel() == 0
    keys = torch.zeros(5000, dtype=torch.int32, device=dev)
    keys[4321] = 1 << 28
    with pytest.raises(pd.PandoraError) as ei:
        pd.sort_pairs(keys, keys.clone(), 28)
    assert ei.value.code == 1   # PANDORA_ERR_INVALID_ARGUMENT
