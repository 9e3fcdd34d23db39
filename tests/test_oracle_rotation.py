"""Pins for the oracle's collision rotation (paper Sec. 2, parts (ii)-(iii)): a particle's
velocity relative to the cell's centre of mass is split along a random axis and the
perpendicular part rotated by the fixed angle alpha.

The rotation is checked against scipy's rotation-vector matrices (an independent
implementation), against closed forms (alpha = 0, pi, rotation about z) and against the
group properties of SO(3).
"""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.spatial.transform import Rotation


def _matrix(orc, n, alpha):
    return np.stack([orc.rotate(n, alpha, np.zeros(3), e) for e in np.eye(3)], axis=1)


def _unit(rng):
    x = rng.standard_normal(3)
    return x / np.linalg.norm(x)


def test_matches_scipy_rotvec(orc):
    rng = np.random.default_rng(7)
    for _ in range(200):
        n = _unit(rng)
        alpha = rng.uniform(-2 * math.pi, 2 * math.pi)
        R = _matrix(orc, n, alpha)
        assert np.allclose(R, Rotation.from_rotvec(alpha * n).as_matrix(), rtol=0, atol=2e-15)


def test_group_properties(orc):
    rng = np.random.default_rng(8)
    for _ in range(100):
        n = _unit(rng)
        a, b = rng.uniform(0, 2 * math.pi, size=2)
        R = _matrix(orc, n, a)
        assert np.abs(R.T @ R - np.eye(3)).max() <= 1e-15 * 4
        assert abs(np.linalg.det(R) - 1.0) < 1e-14
        assert np.allclose(R @ n, n, rtol=0, atol=1e-15 * 4)
        assert np.allclose(_matrix(orc, n, -a) @ R, np.eye(3), rtol=0, atol=1e-15 * 4)
        assert np.allclose(_matrix(orc, n, b) @ R, _matrix(orc, n, a + b), rtol=0, atol=1e-14)


def test_closed_forms(orc):
    c, s = math.cos(1.1), math.sin(1.1)
    Rz = _matrix(orc, np.array([0.0, 0.0, 1.0]), 1.1)
    assert np.allclose(Rz, [[c, -s, 0], [s, c, 0], [0, 0, 1]], rtol=0, atol=1e-16 * 4)
    rng = np.random.default_rng(9)
    for _ in range(50):
        n = _unit(rng)
        v = rng.standard_normal(3)
        u = rng.standard_normal(3)
        assert np.array_equal(orc.rotate(n, 0.0, u, v), u + (v - u)) or np.allclose(
            orc.rotate(n, 0.0, u, v), v, rtol=0, atol=1e-15)
        d = v - u
        flip = u + 2 * np.dot(n, d) * n - d            # rotation by pi
        assert np.allclose(orc.rotate(n, math.pi, u, v), flip, rtol=0, atol=1e-14)
        # the angle between old and new perpendicular parts is alpha, lengths kept
        alpha = 2.2689280275926285  # 130 degrees
        w = orc.rotate(n, alpha, u, v) - u
        perp0 = d - np.dot(n, d) * n
        perp1 = w - np.dot(n, w) * n
        assert abs(np.dot(n, w) - np.dot(n, d)) < 1e-14
        assert abs(np.linalg.norm(perp1) - np.linalg.norm(perp0)) < 1e-14
        cosang = np.dot(perp0, perp1) / (np.linalg.norm(perp0) * np.linalg.norm(perp1))
        assert abs(cosang - math.cos(alpha)) < 1e-12
        # right-hand sense: (perp0 x perp1) points along +n
        assert np.dot(np.cross(perp0, perp1), n) > 0


def test_axis_uniform_on_sphere(orc):
    p = orc.make_params(16)
    ns = np.array([orc.axis(p, t, c) for t in range(1, 6) for c in range(0, 16**3, 1)])
    assert np.abs(np.linalg.norm(ns, axis=1) - 1.0).max() < 4e-16
    N = len(ns)
    assert np.abs(ns.mean(axis=0)).max() < 4.0 / math.sqrt(3 * N)
    second = ns.T @ ns / N
    assert np.abs(second - np.eye(3) / 3).max() < 0.01
    # Archimedes: the z component is uniform on [-1, 1]; the azimuth is uniform
    assert stats.kstest((ns[:, 2] + 1) / 2, "uniform").pvalue > 1e-3
    phi = np.mod(np.arctan2(ns[:, 1], ns[:, 0]), 2 * math.pi) / (2 * math.pi)
    assert stats.kstest(phi, "uniform").pvalue > 1e-3


def test_axis_keyed_by_step_and_cell(orc):
    p = orc.make_params(16, seed=5)
    assert np.array_equal(orc.axis(p, 3, 17), orc.axis(p, 3, 17))
    assert not np.array_equal(orc.axis(p, 3, 17), orc.axis(p, 3, 18))
    assert not np.array_equal(orc.axis(p, 3, 17), orc.axis(p, 4, 17))
