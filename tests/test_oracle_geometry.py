"""Pins for the oracle's random grid shift and cell keys (paper Sec. 2 and Sec. 3.1,
Listing 1: every particle is flagged with the id of the shifted collision cell it sits in).

Keys are checked by brute force on tiny boxes against exact rational arithmetic: with
positions and shifts on a lattice of spacing a/8, floor((r - s)/a) is an exact integer
computation, independent of floating point.
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats


def test_shift_range_and_uniformity(orc):
    p = orc.make_params(16)
    s = np.array([orc.shift(p, t) for t in range(1, 20001)])
    assert s.min() >= -0.5 and s.max() < 0.5
    for d in range(3):
        assert stats.kstest(s[:, d] + 0.5, "uniform").pvalue > 1e-3
    # the three components are independent draws, not copies
    assert abs(np.corrcoef(s[:, 0], s[:, 1])[0, 1]) < 0.03
    # scales with the cell size
    p2 = orc.make_params(16, a=0.5)
    assert np.allclose(np.array([orc.shift(p2, t) for t in range(1, 50)]) * 2.0, s[:49], rtol=0, atol=0)


def test_shift_is_counter_based(orc):
    p = orc.make_params(16, seed=99)
    assert np.array_equal(orc.shift(p, 7), orc.shift(p, 7))
    assert not np.array_equal(orc.shift(p, 7), orc.shift(p, 8))
    q = orc.make_params(16, seed=100)
    assert not np.array_equal(orc.shift(p, 7), orc.shift(q, 7))


def test_shift_walls_folded(orc):
    p = orc.make_params((8, 8, 8), walls_z=1)
    s = np.array([orc.shift(p, t) for t in range(1, 5001)])
    assert s[:, 2].min() >= 0.0 and s[:, 2].max() < 1.0
    assert s[:, :2].min() >= -0.5 and s[:, :2].max() < 0.5


def _exact_key(L, r, s, a, walls=False):
    c = []
    for d in range(3):
        k = math.floor((Fraction(r[d]) - Fraction(s[d])) / Fraction(a))
        if d == 2 and walls:
            c.append(k + 1)
        else:
            c.append(k % L[d])
    return c[0] + L[0] * (c[1] + L[1] * c[2])


@pytest.mark.parametrize("L", [(1, 1, 1), (2, 2, 2), (3, 3, 3), (2, 3, 5)])
@pytest.mark.parametrize("a", [1.0, 0.5])
def test_keys_brute_force(orc, L, a):
    p = orc.make_params(L, a=a)
    box = [Ld * a for Ld in L]
    shifts = [x * a for x in (-0.5, -0.25, -0.125, 0.0, 0.25, 0.375)]
    # every lattice point of spacing a/8 inside the box along each axis, plus the largest
    # double below the box edge
    axes = []
    for d in range(3):
        pts = [k * a / 8 for k in range(8 * L[d])]
        pts.append(np.nextafter(box[d], 0.0))
        axes.append(pts)
    rng = np.random.default_rng(11)
    for sx in shifts:
        for sy in shifts[::2]:
            for sz in shifts[1::2]:
                s = (sx, sy, sz)
                for _ in range(150):
                    r = [axes[d][rng.integers(len(axes[d]))] for d in range(3)]
                    assert orc.cell_key(p, r, s) == _exact_key(L, r, s, a), (r, s)


def test_keys_every_face_point(orc):
    """All 8^3 L^3 lattice points of a 2x2x2 box with one shift: a full enumeration."""
    L = (2, 2, 2)
    p = orc.make_params(L)
    s = (0.25, -0.5, 0.125)
    pts = [k / 8 for k in range(16)]
    for x in pts:
        for y in pts:
            for z in pts:
                assert orc.cell_key(p, (x, y, z), s) == _exact_key(L, (x, y, z), s, 1.0)


def test_zero_shift_is_floor(orc):
    L = (5, 4, 3)
    p = orc.make_params(L)
    rng = np.random.default_rng(3)
    for r in rng.random((500, 3)) * np.array(L):
        c = np.floor(r).astype(int)
        assert orc.cell_key(p, r, (0.0, 0.0, 0.0)) == c[0] + 5 * (c[1] + 4 * c[2])


def test_walls_layers(orc):
    L = (2, 2, 4)
    p = orc.make_params(L, walls_z=1)
    for sz in (0.0, 0.125, 0.5, 0.875):
        for k in range(4 * 8):
            z = k / 8
            key = orc.cell_key(p, (0.0, 0.0, z), (0.0, 0.0, sz))
            assert key == _exact_key(L, (0.0, 0.0, z), (0.0, 0.0, sz), 1.0, walls=True)
            assert 0 <= key // 4 <= 4
    assert orc.num_cells(p) == 2 * 2 * 5


def test_walls_layer_stays_in_range_for_inexact_a(orc):
    """z just below H with a = 0.7, Lz = 5: (z - s)/a rounds to exactly Lz in FP64; the
    layer must still be Lz (the top layer), not Lz + 1."""
    p = orc.make_params((2, 2, 5), a=0.7, walls_z=1)
    H = 5 * 0.7
    z = np.nextafter(H, 0.0)
    assert (z - 0.0) / 0.7 == 5.0        # the rounding that makes this an edge case
    key = orc.cell_key(p, (0.1, 0.1, z), (0.0, 0.0, 0.0))
    assert key // 4 == 5
