"""Pins for the oracle's per-particle masses (reading R24).

The paper's cell sums weight each velocity by its particle's mass (Sec. 3.3, Listing 4:
sum m v and sum m); with one mass per particle, the centre-of-mass velocity is
u = sum m_i v_i / sum m_i, and rotating every v_i - u by the same rotation keeps the cell's
momentum and kinetic energy.  What pins the oracle, independently of its code:
  * a mass array equal to the box mass everywhere reproduces the plain step bit for bit;
  * with random masses, per-cell momentum and kinetic energy are unchanged (numpy);
  * a two-particle cell of unequal masses has a closed form (scipy rotation about the axis);
  * the thermostat gives each cell sum m_i |v_i - u|^2 / 2 = 3/2 (n_c - 1) kT;
  * the angular-momentum correction keeps sum m_i rho_i x v_i about the mass-weighted centre;
  * masses stay with their particles through re-sorts.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2212_11878_gb300 import inputs


def _state(L, seed, ppc=10, lo=0.5, hi=4.0):
    n = int(round(ppc * np.prod(L)))
    r, v = inputs.uniform_gaussian_state(L, n, seed)
    m = np.random.default_rng(seed + 1).uniform(lo, hi, n)
    return r, v, m


def _per_cell(keys, C, x):
    return np.stack([np.bincount(keys, weights=x[:, d], minlength=C) for d in range(3)], axis=1)


@pytest.mark.parametrize("kw", [dict(), dict(thermostat=1, resort_k=2), dict(walls_z=1, g=(0.01, 0.0, 0.0)),
                                dict(thermostat=2, mass=1.7)])
def test_uniform_mass_array_is_the_plain_step(orc, kw):
    L = (6, 5, 4)
    r, v, _ = _state(L, 3)
    p = orc.make_params(L, seed=4, **kw)
    a = orc.State(r, v)
    b = orc.State(r, v, m=np.full(len(r), p.mass))
    for _ in range(3):
        oa = orc.step(p, a, debug=True)
        ob = orc.step(p, b, debug=True)
    assert np.array_equal(a.v, b.v) and np.array_equal(a.r, b.r) and np.array_equal(oa["moments"], ob["moments"])


def test_momentum_and_energy_conserved_per_cell_with_masses(orc):
    L = (7, 6, 5)
    r, v, m = _state(L, 5)
    p = orc.make_params(L, seed=6, dt=0.0)  # dt = 0: the collision alone changes v
    st = orc.State(r, v, m=m)
    out = orc.step(p, st, debug=True)
    keys, C = out["keys"], orc.num_cells(p)
    P0, P1 = _per_cell(keys, C, m[:, None] * v), _per_cell(keys, C, m[:, None] * st.v)
    E0 = np.bincount(keys, weights=0.5 * m * (v * v).sum(axis=1), minlength=C)
    E1 = np.bincount(keys, weights=0.5 * m * (st.v * st.v).sum(axis=1), minlength=C)
    scale = np.bincount(keys, weights=m * np.abs(v).sum(axis=1), minlength=C) + 1e-300
    assert np.all(np.abs(P1 - P0).max(axis=1) <= 1e-12 * scale)
    assert np.all(np.abs(E1 - E0) <= 1e-12 * np.maximum(E0, 1e-300))
    assert np.allclose(out["moments"][:, 0], np.bincount(keys, weights=m, minlength=C), rtol=1e-14)
    assert np.allclose(out["moments"][:, 1:4], P0, rtol=1e-13, atol=1e-13)
    assert np.abs(st.v - v).max() > 0.1  # the collision did something


def test_two_unequal_masses_closed_form(orc):
    p = orc.make_params((1, 1, 1), dt=0.0, ppc=2, alpha_deg=77.0, seed=12)
    r = np.array([[0.125, 0.25, 0.5], [0.75, 0.625, 0.375]])
    v = np.array([[0.3, -1.1, 0.7], [-0.2, 0.4, 1.5]])
    m = np.array([0.7, 3.1])
    st = orc.State(r, v, t=0, m=m)
    orc.step(p, st)
    u = (m[:, None] * v).sum(axis=0) / m.sum()
    R = Rotation.from_rotvec(p.alpha * orc.axis(p, 1, 0)).as_matrix()
    expect = u + (v - u) @ R.T
    assert np.abs(st.v - expect).max() < 1e-14


def test_thermostat_sets_mass_weighted_cell_temperature(orc):
    L = (6, 6, 6)
    r, v, m = _state(L, 7)
    p = orc.make_params(L, thermostat=1, kT=1.4, seed=8)
    st = orc.State(r, v, m=m)
    out = orc.step(p, st, debug=True)
    keys, C = out["keys"], orc.num_cells(p)
    M = np.bincount(keys, weights=m, minlength=C)
    u = _per_cell(keys, C, m[:, None] * st.v) / np.maximum(M, 1e-300)[:, None]
    K = np.bincount(keys, weights=0.5 * m * ((st.v - u[keys]) ** 2).sum(axis=1), minlength=C)
    cnt = np.bincount(keys, minlength=C)
    ok = cnt >= 2
    assert np.allclose(K[ok], 1.5 * (cnt[ok] - 1) * 1.4, rtol=1e-12, atol=0)


def test_angular_momentum_conserved_with_masses(orc):
    L = (6, 5, 5)
    r, v, m = _state(L, 9)
    p = orc.make_params(L, angular=1, dt=0.0, seed=10)
    st = orc.State(r, v, m=m)
    out = orc.step(p, st, debug=True)
    keys, C = out["keys"], orc.num_cells(p)
    q = (st.r - out["shift"]) / p.a
    loc = q - np.floor(q)
    M = np.bincount(keys, weights=m, minlength=C)
    com = _per_cell(keys, C, m[:, None] * loc) / np.maximum(M, 1e-300)[:, None]
    rho = p.a * (loc - com[keys])
    L0 = _per_cell(keys, C, m[:, None] * np.cross(rho, v))
    L1 = _per_cell(keys, C, m[:, None] * np.cross(rho, st.v))
    scale = np.bincount(keys, weights=m * np.linalg.norm(rho, axis=1) * np.abs(v).sum(axis=1), minlength=C) + 1e-300
    assert np.all(np.abs(L1 - L0).max(axis=1) <= 1e-12 * scale)
    P0, P1 = _per_cell(keys, C, m[:, None] * v), _per_cell(keys, C, m[:, None] * st.v)
    assert np.abs(P1 - P0).max() <= 1e-12 * np.abs(m[:, None] * v).sum(axis=1).max() * 40


def test_masses_follow_particles_through_resort(orc):
    L = (5, 5, 5)
    r, v, m = _state(L, 11)
    p = orc.make_params(L, resort_k=1, seed=12)
    st = orc.State(r, v, m=m)
    for _ in range(3):
        orc.step(p, st)
    assert not np.array_equal(st.id, np.arange(len(r)))  # storage was re-ordered
    assert np.array_equal(st.masses_by_id(), m)
