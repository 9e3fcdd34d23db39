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


# ---- R13: virtual particles in the cells cut by a wall ------------------------------------
# A cell of the bottom layer (z below the shift) or of the top layer (z above Lz - 1 + s_z)
# is cut by a wall.  If it holds n_c < ppc real particles it is filled up to ppc with virtual
# particles of the box mass m, at rest on average: their summed momentum is Gaussian with
# variance (ppc - n_c) m kT per component (the equipartition value of that many particles),
# drawn by Box-Muller from Philox counter (t, cell, WALL, 0).  The centre-of-mass velocity of
# the collision is then (m sum v + P_virtual) / (n_c m + (ppc - n_c) m).

def _virtual_fill_expected(p, seed, t, r, v, m, kT, ppc, alpha, L):
    """Velocities after one step with dt = 0, recomputed from the definition above with
    numpy's Philox, Box-Muller written out and scipy's rotation (nothing from the oracle)."""
    from scipy.spatial.transform import Rotation

    import restate

    s = restate.shift(seed, t, walls_z=True)
    keys = []
    for rr in r:
        cx = int(math.floor(rr[0] - s[0])) % L[0]
        cy = int(math.floor(rr[1] - s[1])) % L[1]
        cz = min(max(int(math.floor(rr[2] - s[2])) + 1, 0), L[2])
        keys.append(cx + L[0] * (cy + L[1] * cz))
    keys = np.array(keys)
    out = v.copy()
    filled = set()
    for c in np.unique(keys):
        idx = np.nonzero(keys == c)[0]
        nc = idx.size
        P = m * v[idx].sum(axis=0)
        M = nc * m
        layer = c // (L[0] * L[1])
        fill = (layer == 0 or layer == L[2]) and nc < ppc
        if fill:
            Mv = (ppc - nc) * m
            w = restate.draw(seed, t, int(c), restate.TAG_WALL)
            g0, g1 = restate.box_muller(w[0], w[1])
            g2, _ = restate.box_muller(w[2], w[3])
            P = P + math.sqrt(Mv * kT) * np.array([g0, g1, g2])
            M = M + Mv
            filled.add(int(c))
        if nc < 2 and not fill:
            continue
        u = P / M
        R = Rotation.from_rotvec(alpha * restate.axis(seed, t, int(c))).as_matrix()
        out[idx] = u + (v[idx] - u) @ R.T
    return out, filled, s


def test_virtual_fill_closed_form(orc):
    """Cut cells at both walls with fewer than ppc particles (three, and one), a cut cell
    holding more than ppc, and an interior cell: every velocity after the collision equals
    its value recomputed from the virtual-particle definition (m = 2, kT = 1.7 and a
    fractional ppc, so that a missing mass factor, a wrong variance or a rounded fill
    count shows)."""
    L = (3, 2, 4)
    m, kT, ppc, seed, alpha = 2.0, 1.7, 6.5, 4244, math.radians(100.0)
    p = orc.make_params(L, walls_z=1, dt=0.0, alpha=alpha, mass=m, kT=kT, ppc=ppc, seed=seed)
    import restate
    s = restate.shift(seed, 1, walls_z=True)
    assert 0.1 < s[2] < 0.9, s              # both wall layers are genuinely cut
    rng = np.random.default_rng(11)

    def at(cx, cy, z, k):
        x = (cx + s[0] + 0.5) % L[0] + np.linspace(-0.3, 0.3, k)
        y = (cy + s[1] + 0.5) % L[1] + np.linspace(0.2, -0.2, k)
        return np.stack([np.mod(x, L[0]), np.mod(y, L[1]), np.full(k, z)], axis=1)

    bottom = 0.5 * s[2]                     # layer 0: z in [0, s_z)
    top = 0.5 * ((L[2] - 1 + s[2]) + L[2])  # layer Lz: z in [Lz - 1 + s_z, Lz)
    interior = 1.5 + s[2]                   # layer 2
    r = np.concatenate([at(0, 0, bottom, 3), at(1, 1, top, 3), at(2, 0, bottom, 1), at(0, 1, top, 7),
                        at(1, 0, interior, 3)])
    v = rng.normal(0.0, 1.0, r.shape) + np.array([0.4, -0.2, 0.1])
    st = orc.State(r, v)
    orc.step(p, st)
    _, vr = st.by_id()
    expect, filled, _ = _virtual_fill_expected(p, seed, 1, r, v, m, kT, ppc, alpha, L)
    assert len(filled) == 3                 # the two three-particle cells and the lone particle
    assert np.abs(vr - expect).max() < 1e-13, np.abs(vr - expect).max()
    # the interior cell and the over-full cut cell are the plain collision (no fill)
    assert not np.allclose(vr[-3:], v[-3:])


def test_virtual_fill_only_in_cut_layers_and_variance(orc):
    """One particle at rest in every cell, dt = 0, alpha = 180 degrees.  Interior cells hold a
    single particle and no virtual ones, so nothing changes there.  In a cut cell the
    collision gives v' = u + R(0 - u) = 2 u_perp, with u = P_virtual / (ppc m), hence
    <|v'|^2> = (8/3) <|u|^2> = 8 (ppc - 1) kT / (ppc^2 m) over steps and cells, and the mean
    of v' is zero."""
    import restate

    L = (6, 6, 3)
    m, kT, ppc, seed = 2.0, 1.3, 5.5, 99
    p = orc.make_params(L, walls_z=1, dt=0.0, alpha=math.pi, mass=m, kT=kT, ppc=ppc, seed=seed)
    samples = []
    for t in range(1, 151):
        s = restate.shift(seed, t, walls_z=True)
        xs = (np.arange(L[0]) + s[0] + 0.5) % L[0]
        ys = (np.arange(L[1]) + s[1] + 0.5) % L[1]
        zs = [0.5 * s[2]] + [k + s[2] - 0.5 for k in range(1, L[2])] + [0.5 * ((L[2] - 1 + s[2]) + L[2])]
        grid = np.array([[x, y, z] for z in zs for y in ys for x in xs])
        st = orc.State(grid, np.zeros_like(grid), t=t - 1)
        orc.step(p, st)
        _, vr = st.by_id()
        layer = np.repeat(np.arange(L[2] + 1), L[0] * L[1])
        cut = (layer == 0) | (layer == L[2])
        assert np.all(vr[~cut] == 0.0), t   # no virtual particles in the interior
        assert np.all(np.abs(vr[cut]).sum(axis=1) > 0.0), t
        samples.append(vr[cut])
    vv = np.concatenate(samples)
    expect = 8.0 * (ppc - 1.0) * kT / (ppc * ppc * m)
    got = (vv * vv).sum(axis=1).mean()
    assert abs(got / expect - 1.0) < 0.05, (got, expect)
    sem = math.sqrt(expect / 3.0 / len(vv))
    assert np.all(np.abs(vv.mean(axis=0)) < 5.0 * sem)
