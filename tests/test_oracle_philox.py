"""Pins for the oracle's Philox4x64-10 and its uniform mapping.

Philox4x64-10 is the counter-based generator of Salmon et al. (SC'11) that the oracle uses
for every random draw (grid shift, rotation axis, initial state).  Pinned against the
published known-answer vector and against numpy's independent Philox implementation.
"""
import os

import numpy as np
import pytest

from restate import philox as _numpy_philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        left, right = line.split("->")
        words = [int(w, 16) for w in left.split()]
        out = [int(w, 16) for w in right.split()]
        rows.append((words[:4], words[4:6], out))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_published_kat(orc, ctr, key, expect):
    assert [int(x) for x in orc.philox(ctr, key)] == expect


def test_matches_numpy_philox(orc):
    rng = np.random.default_rng(1234)
    cases = []
    for _ in range(300):
        ctr = [int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)) for _ in range(4)]
        key = [int(rng.integers(0, 2**63)) * 2 + int(rng.integers(0, 2)) for _ in range(2)]
        cases.append((ctr, key))
    # counters whose low word is zero (the numpy start needs a borrow) and the counter
    # layouts the method uses: (t, 0, SHIFT, 0), (t, cell, AXIS, 0), (i, j, INIT, 0)
    cases += [([0, 5, 1, 0], [7, 0]), ([0, 0, 0, 1], [1, 2]), ([2**64 - 1] * 4, [2**64 - 1] * 2)]
    cases += [([t, 0, 1, 0], [20221211, 0]) for t in range(1, 20)]
    cases += [([3, c, 2, 0], [20221211, 0]) for c in range(0, 4096, 97)]
    for ctr, key in cases:
        assert [int(x) for x in orc.philox(ctr, key)] == _numpy_philox(ctr, key), (ctr, key)


def test_u53_exact_and_in_range(orc):
    assert orc.u53(0) == 0.0
    assert orc.u53(2**64 - 1) == 1.0 - 2.0**-53
    assert orc.u53(1 << 11) == 2.0**-53
    assert orc.u53((1 << 11) - 1) == 0.0          # the low 11 bits are dropped
    assert orc.u53(1 << 63) == 0.5
    rng = np.random.default_rng(5)
    for w in rng.integers(0, 2**63, size=1000, dtype=np.int64):
        w = int(w) * 2 + 1
        x = orc.u53(w)
        assert 0.0 <= x < 1.0
        assert x * 2.0**53 == float(w >> 11)      # exactly k * 2^-53
