"""Helpers shared by the GPU parity tests: running the oracle beside the library from the
same state and comparing results with the stated tolerances.

Tolerances (FP64 form): cell keys, counts, offsets, perm and ids bit-exact; positions and
velocities within 1e-12 relative, per particle:
    |v_gpu - v_ref|_inf <= 1e-12 * max(|v_ref|_inf, sqrt(kT/m))
    periodic |r_gpu - r_ref|_inf <= 1e-12 * max(|r_ref|_inf, a)
The floors keep the bound relative to the physical scales (thermal speed, cell size) for
components that happen to be near zero.
"""
import math

import numpy as np

from paper_2212_11878_gb300 import abi

TOL = 1e-12


def oracle_params(orc, p: abi.Params):
    return orc.make_params(tuple(p.L), a=p.a, dt=p.dt, alpha=p.alpha, kT=p.kT, mass=p.mass, ppc=p.ppc,
                           seed=p.seed, resort_k=p.resort_k, walls_z=p.walls_z, g=tuple(p.g),
                           thermostat=p.thermostat, angular=p.angular)


def periodic_diff(a, b, box, walls_z=False):
    d = np.abs(a - b)
    for k in range(3):
        if k == 2 and walls_z:
            continue
        d[:, k] = np.minimum(d[:, k], box[k] - d[:, k])
    return d


def assert_state_close(r_gpu, v_gpu, r_ref, v_ref, p: abi.Params, tol=TOL, what="", r_scale=None):
    """r_scale: an extra per-particle length scale for the position bound (a particle that
    crosses the box many times per step carries its velocity's rounding times dt)."""
    box = np.array(p.L, dtype=float) * p.a
    sig = math.sqrt(p.kT / p.mass)
    if len(r_ref) == 0:
        assert len(r_gpu) == 0
        return
    dr = periodic_diff(r_gpu, r_ref, box, bool(p.walls_z)).max(axis=1)
    bound_r = tol * np.maximum(np.abs(r_ref).max(axis=1), p.a)
    if r_scale is not None:
        bound_r = np.maximum(bound_r, tol * r_scale)
    dv = np.abs(v_gpu - v_ref).max(axis=1)
    bound_v = tol * np.maximum(np.abs(v_ref).max(axis=1), sig)
    bad_r = np.nonzero(dr > bound_r)[0]
    bad_v = np.nonzero(dv > bound_v)[0]
    assert bad_r.size == 0, "%s positions: %d particles off, worst %g (particle %d)" % (
        what, bad_r.size, (dr / bound_r).max(), int(np.argmax(dr / bound_r)))
    assert bad_v.size == 0, "%s velocities: %d particles off, worst ratio %g (particle %d)" % (
        what, bad_v.size, (dv / bound_v).max(), int(np.argmax(dv / bound_v)))


def assert_sort_equal(dbg_gpu, dbg_ref):
    for k in ("keys", "counts", "offsets", "perm", "ids"):
        a, b = dbg_gpu[k], dbg_ref[k]
        assert a.shape == b.shape, k
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError("%s differs at %d entries, first %d: gpu %d oracle %d" % (
                k, bad.size, bad[0], a[bad[0]], b[bad[0]]))


def face_distance(r, s, a=1.0):
    """Distance (cell units) of each position from the nearest face of the grid shifted by s."""
    x = (r - s) / a
    fr = x - np.floor(x)
    return np.minimum(fr, 1 - fr).min(axis=1)


def assert_mixed_one_step(p, kg, ko, rg, vg, rr, vr, shift, ncell, what=""):
    """Bounds of one mixed-form step from a state both forms represent exactly, against the
    FP64 oracle (all arrays by particle id; kg, ko the cell keys of the GPU and the oracle):
      - key disagreements are rare (at most 2e-5 of the particles, or 3) and each lies within
        1e-5 cells of a shifted cell face (FP32 positions round across the face);
      - positions within 1e-6 relative (periodic distance);
      - velocities, in cells without a key disagreement, within 5e-6 of max(|v|, sqrt(kT/m))."""
    n = len(kg)
    bad = np.nonzero(kg != ko)[0]
    assert bad.size <= max(3, 2e-5 * n), "%s: %d key disagreements" % (what, bad.size)
    if bad.size:
        assert face_distance(rr[bad], shift, p.a).max() < 1e-5, what
    L = tuple(p.L)
    box_len = np.array(L, float) * p.a
    assert (periodic_diff(rg, rr, box_len, bool(p.walls_z)).max(axis=1)
            <= 1e-6 * np.maximum(np.abs(rr).max(axis=1), p.a)).all(), what
    clean_cells = np.setdiff1d(np.arange(ncell), np.concatenate([kg[bad], ko[bad]]))
    clean = np.isin(ko, clean_cells)
    sig = math.sqrt(p.kT / p.mass)
    dv = np.abs(vg - vr).max(axis=1)[clean]
    assert (dv <= 5e-6 * np.maximum(np.abs(vr).max(axis=1)[clean], sig)).all(), (what, dv.max())
