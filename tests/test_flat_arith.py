"""The exact stability sums of the flat-cluster kernels, checked on the CPU.

csrc/flat.cu's digit split (split_digits) and its round-once conversion
(round_fixed) are host-callable; this test compiles them from the library
source into a small host program (nvcc, no GPU needed), accumulates groups of
float64 terms the way the kernels do (one digit triple per term, times its
multiplicity, into 64-bit words; carries; rounding), and compares every
result with Python's exact rational sum rounded once.  Terms are built as the
kernels build them: differences of lambdas 1/w of float32 weights, times
multiplicities whose total stays below 2^29 per group.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FLAT_CU = os.path.join(ROOT, "paper_2401_06089_gb300", "csrc", "flat.cu")

HARNESS = r"""
#include "%s"
#include <cstdio>
namespace pandora { cudaMemPool_t flat_pool(int) { return nullptr; } }
int main()
{
    char buf[256];
    u64 acc[NL] = {0};
    bool bad = false;
    while (fgets(buf, sizeof buf, stdin)) {
        if (buf[0] == 'E') {
            u32 D[NL];
            u64 carry = 0;
            for (int j = 0; j < NL; ++j) {
                const u64 v = acc[j] + carry;
                D[j] = (u32)v;
                carry = v >> 32;
                acc[j] = 0;
            }
            printf("%%a %%d %%d\n", round_fixed(D), (int)(carry != 0), (int)bad);
            bad = false;
            continue;
        }
        unsigned long long mult;
        double t;
        if (sscanf(buf, "%%llu %%la", &mult, &t) != 2)
            return 2;
        int j0;
        u32 d[3];
        if (split_digits(t, j0, d[0], d[1], d[2], bad))
            for (int q = 0; q < 3; ++q)
                acc[j0 + q] += (u64)d[q] * mult;
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("flat_arith")
    src = d / "harness.cu"
    exe = d / "harness"
    src.write_text(HARNESS % FLAT_CU)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-o", str(exe), str(src)], check=True, capture_output=True)
    return str(exe)


def _run(exe, groups):
    lines = []
    for g in groups:
        lines += [f"{m} {t.hex()}" for m, t in g] + ["END"]
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    res = []
    for o in out[:len(groups)]:
        r, carry, bad = o.split()
        res.append((float.fromhex(r), int(carry), int(bad)))
    return res


def _exact(g):
    s = sum((m * Fraction(t) for m, t in g), Fraction(0))
    return s.numerator / s.denominator


def test_random_groups_equal_exact_sum_rounded_once(harness):
    rng = np.random.default_rng(1)
    groups = []
    for k in range(6000):
        kind = k % 5
        cnt = int(rng.integers(1, 60))
        if kind == 0:
            w = rng.uniform(0.5, 2.0, size=(cnt, 2)).astype(np.float32)
        elif kind == 1:      # the whole float32 range
            w = np.exp2(rng.uniform(-149, 127, size=(cnt, 2))).astype(np.float32)
            w[w == 0] = np.float32(2.0 ** -149)
        elif kind == 2:      # neighbouring weights: tiny differences
            base = rng.uniform(1, 2, size=cnt).astype(np.float32)
            w = np.stack([base, np.nextafter(base, np.float32(3))], 1)
        elif kind == 3:      # powers of two: exact halfway cases
            w = np.exp2(rng.integers(-20, 20, size=(cnt, 2))).astype(np.float32)
        else:
            w = np.exp2(rng.uniform(-60, 60, size=(cnt, 2))).astype(np.float32)
        g = []
        for a, b in w:
            la, lb = 1.0 / float(a), 1.0 / float(b)
            hi, lo = max(la, lb), min(la, lb)
            if rng.random() < 0.2:
                lo = 0.0
            mult = int(rng.integers(1, 2 ** 29 // 64)) if rng.random() < 0.3 else 1
            g.append((mult, hi - lo))
        groups.append(g)
    for g, (got, carry, bad) in zip(groups, _run(harness, groups)):
        assert carry == 0 and bad == 0
        assert got == _exact(g)


def test_boundaries_and_ties_to_even(harness):
    groups = [
        [(1, 1.0), (1, 2.0 ** -53)],                       # halfway, rounds to even (down)
        [(1, 1.0 + 2.0 ** -52), (1, 2.0 ** -53)],          # halfway, rounds to even (up)
        [(1, 1.0), (1, 2.0 ** -53), (1, 2.0 ** -180)],     # just above halfway
        [(3, 2.0 ** -180)],                                # the smallest unit
        [(1, 2.0 ** 149), (2 ** 28, 2.0 ** 149)],          # the largest terms
        [(1, 0.0)],
        [(1, 2.0 ** -128 - 2.0 ** -180)],
        [(1, (2 - 2.0 ** -52) * 2.0 ** 148)] * 2,          # carry into a new exponent
        [(5, 2.0 ** -53), (1, 1.0)],
    ]
    for g, (got, carry, bad) in zip(groups, _run(harness, groups)):
        assert carry == 0 and bad == 0
        assert got == _exact(g), g


def test_terms_outside_the_exact_form_are_flagged(harness):
    """A negative term, a subnormal, and a value finer than 2^-180 are not
    sums the kernels can take exactly: the split reports them."""
    for t in (-1.0, 5e-324, 2.0 ** -200 * 3):
        (_, _, bad), = _run(harness, [[(1, t)]])
        assert bad == 1, t
