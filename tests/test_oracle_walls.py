"""Pins for the oracle's channel-flow extension: bounce-back walls at z = 0 and z = H with
virtual particles in cut cells, a constant body force along x and the cell-level
thermostat.  The paper's benchmark fluid is periodic (Sec. 4); these parts follow the
standard SRD no-slip construction that its MPCD reference describes.

Pins: the bounce-back closed form for one particle, confinement, and the steady Poiseuille
profile v_x(z) = g z (H - z) / (2 nu) with the SRD kinematic viscosity nu = nu_kin + nu_coll
(mean-field formulas for 3-D SRD with random shift).
"""
import math

import numpy as np

from paper_2212_11878_gb300 import inputs


def srd_viscosity(n, alpha, dt, kT=1.0, m=1.0, a=1.0):
    """Kinematic viscosity of 3-D SRD with random grid shift (kinetic + collisional parts)."""
    f = n - 1.0 + math.exp(-n)
    nu_kin = kT * dt / (2.0 * m) * (5.0 * n / (f * (2.0 - math.cos(alpha) - math.cos(2.0 * alpha))) - 1.0)
    nu_col = a * a / (18.0 * dt) * (f / n) * (1.0 - math.cos(alpha))
    return nu_kin + nu_col


def test_viscosity_formula_values():
    # n = 20, alpha = 130 deg, dt = 0.1: kinetic ~0.0434, collisional ~0.867 per unit density
    nu = srd_viscosity(20, math.radians(130), 0.1)
    assert abs(20 * nu - 18.2) < 0.1


def test_bounce_back_single_particle(orc):
    L = (4, 4, 4)
    p = orc.make_params(L, walls_z=1, alpha=0.0, dt=0.1)
    r = np.array([[1.3, 2.2, 0.05]])
    v = np.array([[0.3, 0.2, -1.0]])
    st = orc.State(r, v)
    orc.step(p, st)
    # crossing at tau = dt / 2: back at the start point with the velocity reversed
    assert np.allclose(st.r[0], [1.3, 2.2, 0.05], rtol=0, atol=1e-15)
    assert np.allclose(st.v[0], [-0.3, -0.2, 1.0], rtol=0, atol=1e-15)
    # top wall, with a body force along x
    p = orc.make_params(L, walls_z=1, alpha=0.0, dt=0.1, g=(0.5, 0.0, 0.0))
    st = orc.State(np.array([[1.0, 1.0, 3.98]]), np.array([[0.0, 0.0, 0.5]]))
    orc.step(p, st)
    tau = 0.04
    vx_hit = 0.5 * tau
    x_hit = 1.0 + 0.25 * tau * tau
    rest = 0.1 - tau
    assert np.allclose(st.r[0], [x_hit - vx_hit * rest + 0.25 * rest * rest, 1.0, 4.0 - 0.5 * rest],
                       rtol=0, atol=1e-14)
    assert np.allclose(st.v[0], [-vx_hit + 0.5 * rest, 0.0, -0.5], rtol=0, atol=1e-14)


def test_confined_and_layers(orc):
    L = (6, 5, 7)
    p = orc.make_params(L, walls_z=1, ppc=10, dt=0.5, g=(0.01, 0, 0))
    n = 10 * 6 * 5 * 7
    r, v = inputs.uniform_gaussian_state(L, n, 3)
    st = orc.State(r, v * 3.0)
    for _ in range(20):
        out = orc.step(p, st, debug=True)
        assert np.all(st.r[:, 2] >= 0.0) and np.all(st.r[:, 2] < 7.0)
        layers = out["keys"] // (6 * 5)
        assert layers.min() >= 0 and layers.max() <= 7


def test_poiseuille_profile(orc):
    Lx, Ly, H = 6, 6, 10
    n_bar, g, dt, alpha = 10, 0.01, 0.1, math.radians(130)
    p = orc.make_params((Lx, Ly, H), walls_z=1, ppc=n_bar, dt=dt, alpha=alpha, g=(g, 0.0, 0.0),
                        thermostat=1, seed=77)
    n = n_bar * Lx * Ly * H
    r, v = inputs.uniform_gaussian_state((Lx, Ly, H), n, 77)
    st = orc.State(r, v)
    nu = srd_viscosity(n_bar, alpha, dt)
    tau_relax = H * H / (math.pi ** 2 * nu)            # slowest mode of the start-up flow
    burn = int(6 * tau_relax / dt)
    avg_steps = 5000
    orc.run(p, st, burn)
    nb = 10
    acc = np.zeros(nb)
    cnt = np.zeros(nb)
    for _ in range(avg_steps):
        orc.step(p, st)
        b = np.minimum((st.r[:, 2] / H * nb).astype(int), nb - 1)
        acc += np.bincount(b, weights=st.v[:, 0], minlength=nb)
        cnt += np.bincount(b, minlength=nb)
    prof = acc / cnt
    z = (np.arange(nb) + 0.5) * H / nb
    # free quadratic fit v = c0 + c1 z + c2 z^2; Poiseuille has c2 = -g / (2 nu)
    A = np.stack([np.ones(nb), z, z * z], axis=1)
    coef, *_ = np.linalg.lstsq(A, prof, rcond=None)
    resid = prof - A @ coef
    r2 = 1 - (resid ** 2).sum() / ((prof - prof.mean()) ** 2).sum()
    assert r2 > 0.98
    nu_fit = -g / (2 * coef[2])
    assert abs(nu_fit / nu - 1) < 0.12, (nu_fit, nu)
    vmax = g * H * H / (8 * nu)
    vertex = -coef[1] / (2 * coef[2])
    assert abs(vertex - H / 2) < 0.05 * H              # symmetric between the walls
    assert abs(coef[0]) < 0.15 * vmax                  # little slip at z = 0
    assert abs(coef[0] + coef[1] * H + coef[2] * H * H) < 0.15 * vmax  # and at z = H
