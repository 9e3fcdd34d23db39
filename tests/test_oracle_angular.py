"""Pins for the oracle's angular-momentum-conserving collision (reading R23).

The plain SRD rotation conserves each cell's momentum and kinetic energy but not its angular
momentum.  The variant that the paper mentions (Sec. 2, from the Gompper et al. review it
cites) adds omega x rho_i to every member after the rotation, with rho_i the particle's
position relative to the cell's centre of mass and omega = I^-1 (L_before - L_after), I the
cell's inertia tensor.

What pins it, independently of the oracle's code:
  * per cell, the angular momentum about the centre of mass (computed here with numpy from
    positions on the shifted grid) and the momentum are unchanged by the collision;
  * a two-particle cell has a closed form: the relative velocity keeps its part normal to the
    separation and takes the component along it from the rotated relative velocity (scipy
    rotation about the cell's axis);
  * in every cell the result equals the plain collision (same step, variant off) plus
    omega x rho_i with omega from LAPACK's solve (or pseudo-inverse for two particles);
  * alpha = 0 changes nothing; a cell of collinear particles gets no correction.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2212_11878_gb300 import inputs


def _step_pair(orc, L, seed, **kw):
    """One step with and without the variant from the same state (no force: streaming leaves
    the velocities alone, so the pre-collision velocities are the initial ones)."""
    n = int(round(kw.pop("ppc", 10) * np.prod(L)))
    r, v = inputs.uniform_gaussian_state(L, n, seed)
    outs = {}
    for ang in (0, 1):
        p = orc.make_params(L, angular=ang, seed=seed + 100, **kw)
        st = orc.State(r, v)
        out = orc.step(p, st, debug=True)
        outs[ang] = (p, st, out)
    return r, v, outs


def _rho(p, r_streamed, shift, keys, C):
    q = (r_streamed - shift) / p.a
    loc = q - np.floor(q)
    cnt = np.bincount(keys, minlength=C)
    mean = np.stack([np.bincount(keys, weights=loc[:, d], minlength=C) for d in range(3)], axis=1)
    mean /= np.maximum(cnt, 1)[:, None]
    return p.a * (loc - mean[keys]), cnt


def _per_cell(keys, C, x):
    return np.stack([np.bincount(keys, weights=x[:, d], minlength=C) for d in range(3)], axis=1)


@pytest.mark.parametrize("thermostat", [0, 1, 2])
def test_angular_momentum_and_momentum_conserved_per_cell(orc, thermostat):
    L = (7, 6, 5)
    r0, v0, outs = _step_pair(orc, L, 3, thermostat=thermostat, mass=1.3)
    p, st, out = outs[1]
    C = orc.num_cells(p)
    keys = out["keys"]
    rho, cnt = _rho(p, st.r, out["shift"], keys, C)
    m = p.mass
    Lb = m * _per_cell(keys, C, np.cross(rho, v0))
    La = m * _per_cell(keys, C, np.cross(rho, st.v))
    scale = m * np.bincount(keys, weights=np.linalg.norm(rho, axis=1) * np.abs(v0).sum(axis=1), minlength=C) + 1e-300
    assert np.all(np.abs(La - Lb).max(axis=1) <= 1e-12 * scale)
    Pb = _per_cell(keys, C, v0)
    Pa = _per_cell(keys, C, st.v)
    assert np.abs(Pa - Pb).max() <= 1e-12 * np.abs(v0).sum(axis=1).max() * cnt.max()
    if thermostat == 0:
        # the plain rotation alone would not conserve it: the pin is not vacuous
        p0, st0, _ = outs[0]
        L0 = m * _per_cell(keys, C, np.cross(rho, st0.v))
        assert np.abs(L0 - Lb).max() > 1e-3


def test_correction_equals_plain_collision_plus_omega_cross_rho(orc):
    L = (6, 6, 6)
    r0, v0, outs = _step_pair(orc, L, 5, thermostat=1, kT=1.2)
    p, st, out = outs[1]
    _, st0, out0 = outs[0]
    assert np.array_equal(out["keys"], out0["keys"])
    C = orc.num_cells(p)
    keys = out["keys"]
    rho, cnt = _rho(p, st.r, out["shift"], keys, C)
    m = p.mass
    dL = m * (_per_cell(keys, C, np.cross(rho, v0)) - _per_cell(keys, C, np.cross(rho, st0.v)))
    expect = st0.v.copy()
    for c in np.nonzero(cnt >= 2)[0]:
        idx = np.nonzero(keys == c)[0]
        q = rho[idx]
        I = m * ((q * q).sum() * np.eye(3) - q.T @ q)
        w = np.linalg.pinv(I) @ dL[c] if len(idx) == 2 else np.linalg.solve(I, dL[c])
        expect[idx] += np.cross(w, q)
    err = np.abs(st.v - expect).max(axis=1)
    assert np.all(err <= 1e-10 * np.maximum(np.abs(expect).max(axis=1), 1.0))


def test_two_particle_cell_closed_form(orc):
    L = (1, 1, 1)
    p = orc.make_params(L, angular=1, dt=0.0, ppc=2, alpha_deg=107.0, seed=9)
    r = np.array([[0.125, 0.25, 0.5], [0.75, 0.625, 0.375]])
    v = np.array([[0.3, -1.1, 0.7], [-0.2, 0.4, 1.5]])
    st = orc.State(r, v, t=0)
    out = orc.step(p, st, debug=True)
    loc = np.array([orc.cell_local(p, x, out["shift"]) for x in r])
    e = loc[0] - loc[1]
    e /= np.linalg.norm(e)
    n = orc.axis(p, 1, 0)
    R = Rotation.from_rotvec(p.alpha * n).as_matrix()
    u = v.mean(axis=0)
    w = v[0] - v[1]
    w_new = w - (w @ e) * e + ((R @ w) @ e) * e
    expect = np.stack([u + 0.5 * w_new, u - 0.5 * w_new])
    assert np.abs(st.v - expect).max() < 1e-14


def test_alpha_zero_changes_nothing(orc):
    L = (5, 5, 5)
    r0, v0, outs = _step_pair(orc, L, 7, alpha=0.0)
    assert np.abs(outs[1][1].v - v0).max() < 1e-14


def test_collinear_cell_is_not_corrected(orc):
    L = (1, 1, 1)
    r = np.array([[0.125, 0.5, 0.5], [0.5, 0.5, 0.5], [0.875, 0.5, 0.5]])
    v = np.array([[0.3, -1.1, 0.7], [-0.2, 0.4, 1.5], [0.9, 0.1, -0.6]])
    res = {}
    for ang in (0, 1):
        p = orc.make_params(L, angular=ang, dt=0.0, ppc=3, seed=10)
        st = orc.State(r, v, t=0)
        orc.step(p, st)
        res[ang] = st.v
    assert np.array_equal(res[0], res[1])


def test_walls_rejected(orc):
    p = orc.make_params((4, 4, 4), angular=1, walls_z=1)
    r, v = inputs.uniform_gaussian_state((4, 4, 4), 640, 1)
    with pytest.raises(Exception):
        orc.step(p, orc.State(r, v))
