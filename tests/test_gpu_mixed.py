"""GPU checks of the mixed-precision form (int32 cell + FP32 offset positions, FP32
velocities, exact/compensated per-cell sums, energy-conserving rescale).

Its trajectories cannot match the FP64 oracle bit for bit: a particle within FP32 rounding
of a shifted cell face can land in the neighbouring cell.  So the checks are
  * one step from a state both forms represent exactly: key disagreements are rare and
    each lies within 1e-5 cells of a face; positions within 1e-6 and velocities (in cells
    without a disagreement) within 5e-6 relative of the oracle;
  * the sort is bit-exact against its own keys (counts, offsets, stable perm);
  * per-cell momentum and energy are conserved to FP32 rounding; energy does not drift;
  * velocity statistics agree with the oracle's; checkpoints resume bit-exactly;
  * Poiseuille flow between walls matches the closed form.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2212_11878_gb300 import abi, inputs
from parity import oracle_params, periodic_diff

pytestmark = pytest.mark.gpu


def quantize(r, v, L, a=1.0):
    """A state the mixed form stores exactly: r = (c + f) a with f an FP32 in [0, 1)."""
    L = np.asarray(L)
    q = r / a
    c = np.floor(q)
    f = (q - c).astype(np.float32).astype(np.float64)
    up = f >= 1.0
    f[up] = 0.0
    c[up] += 1
    c = np.mod(c, L)
    return (c + f) * a, v.astype(np.float32).astype(np.float64)


def mixed_params(L, **kw):
    kw.setdefault("precision", "mixed")
    return abi.make_params(L, **kw)


def face_distance(r, s, a=1.0):
    x = (r - s) / a
    fr = x - np.floor(x)
    return np.minimum(fr, 1 - fr).min(axis=1)


def test_state_roundtrip_exact():
    L = (7, 6, 5)
    p = mixed_params(L)
    n = int(round(p.ppc * 7 * 6 * 5))
    r, v = quantize(*inputs.uniform_gaussian_state(L, n, 3), L)
    with abi.Box(p) as box:
        box.set_state(r, v, 0)
        rg, vg = box.state()
    assert np.array_equal(rg, r) and np.array_equal(vg, v)


def test_init_matches_oracle_to_fp32(orc):
    p = mixed_params((8, 8, 8), seed=11)
    with abi.Box(p) as box:
        rg, vg = box.state()
    rr, vr = orc.init(oracle_params(orc, p), rg.shape[0])
    assert np.abs(rg - rr).max() <= 2 ** -24
    assert np.all(np.abs(vg - vr) <= 2 ** -23 * np.maximum(np.abs(vr), 1e-3))


@pytest.mark.parametrize("case", [dict(L=(12, 10, 8)), dict(L=(9, 9, 9), a=0.5, dt=0.2),
                                  dict(L=(8, 8, 8), g=(0.01, 0.02, -0.01)), dict(L=(8, 7, 6), ppc=25),
                                  dict(L=(10, 9, 8), fast=0.02), dict(L=(9, 8, 7), g=(0.02, 0.0, 0.01), fast=0.01),
                                  dict(L=(10, 9, 8), thermostat=1, kT=1.3), dict(L=(11, 9, 8), thermostat=2, kT=1.3),
                                  dict(L=(9, 8, 10), walls_z=1, g=(0.02, 0.01, 0.0)),
                                  dict(L=(8, 9, 12), walls_z=1, g=(0.01, 0.0, 0.0), thermostat=2, ppc=15),
                                  dict(L=(8, 8, 6), walls_z=1, g=(0.02, 0.0, 0.0), dt=0.3, fast=0.02),
                                  dict(L=(10, 9, 8), angular=1), dict(L=(9, 8, 7), angular=1, thermostat=1, fast=0.01)])
def test_one_step_against_fp64_oracle(orc, case):
    """`fast`: that fraction of the particles moves 0.6 to 3 cells in the step, so that the
    warps holding them take the general carry path instead of the one-cell one.  With walls,
    warps whose particles all stay clear of the walls take the same one-cell path; the others
    bounce in the general loop."""
    case = dict(case)
    fast = case.pop("fast", 0.0)
    p = mixed_params(seed=5, **case)
    L = tuple(p.L)
    n = int(round(p.ppc * np.prod(L)))
    r0, v0 = inputs.uniform_gaussian_state(L, n, 21, a=p.a)
    if fast:
        rng = np.random.default_rng(77)
        ids = rng.choice(n, max(1, int(fast * n)), replace=False)
        speed = rng.uniform(0.6, 3.0, ids.size) * p.a / p.dt
        v0[ids] *= (speed / np.linalg.norm(v0[ids], axis=1))[:, None]
    r0, v0 = quantize(r0, v0, L, p.a)
    with abi.Box(p) as box:
        box.set_state(r0, v0, 4)
        box.step(1)
        dbg = box.debug_sort()
        rg, vg = box.state()
    st = orc.State(r0, v0, t=4)
    ref = orc.step(oracle_params(orc, p), st, debug=True)
    rr, vr = st.by_id()
    # the sort, bit-exact against the GPU's own keys
    C = int(np.prod(L)) if not p.walls_z else L[0] * L[1] * (L[2] + 1)
    keys = dbg["keys"]
    assert np.array_equal(dbg["counts"], np.bincount(keys, minlength=C))
    assert dbg["offsets"][0] == 0 and np.array_equal(dbg["offsets"][1:], np.cumsum(dbg["counts"]))
    assert np.array_equal(dbg["perm"], np.argsort(keys, kind="stable"))
    # keys against the oracle, by particle id
    kg = np.empty(n, np.int64)
    kg[dbg["ids"]] = keys
    ko = np.empty(n, np.int64)
    ko[ref["ids"]] = ref["keys"]
    bad = np.nonzero(kg != ko)[0]
    assert bad.size <= max(3, 2e-5 * n), bad.size
    if bad.size:
        assert face_distance(rr[bad], ref["shift"], p.a).max() < 1e-5
    # positions and velocities
    box_len = np.array(L, float) * p.a
    assert (periodic_diff(rg, rr, box_len).max(axis=1) <= 1e-6 * np.maximum(np.abs(rr).max(axis=1), p.a)).all()
    clean_cells = np.setdiff1d(np.arange(C), np.concatenate([kg[bad], ko[bad]]))
    clean = np.isin(ko, clean_cells)
    sig = math.sqrt(p.kT / p.mass)
    dv = np.abs(vg - vr).max(axis=1)[clean]
    assert (dv <= 5e-6 * np.maximum(np.abs(vr).max(axis=1)[clean], sig)).all(), dv.max()


def test_cell_conservation():
    L = (10, 10, 10)
    p = mixed_params(L, seed=9)
    n = int(round(10 * 1000))
    r0, v0 = quantize(*inputs.uniform_gaussian_state(L, n, 4), L)
    with abi.Box(p) as box:
        box.set_state(r0, v0, 0)
        abi.mpcd_record_moments(box.h, True)
        box.step(1)
        mom, _ = box.moments()
        dbg = box.debug_sort()
        rg, vg = box.state()
    keys = np.empty(n, np.int64)
    keys[dbg["ids"]] = dbg["keys"]
    C = 1000
    P = np.stack([np.bincount(keys, weights=vg[:, d], minlength=C) for d in range(3)], axis=1)
    E = 0.5 * np.bincount(keys, weights=(vg * vg).sum(axis=1), minlength=C)
    scale = np.bincount(keys, weights=np.abs(vg).sum(axis=1), minlength=C) + 1e-30
    assert np.all(np.abs(P - mom[:, 1:4]).max(axis=1) <= 2e-6 * scale)
    assert np.all(np.abs(E - mom[:, 4]) <= 2e-6 * np.maximum(mom[:, 4], 1e-30))
    assert np.array_equal(mom[:, 0], np.bincount(keys, minlength=C).astype(float))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_mbs_thermostat_gives_canonical_cell_energies(precision):
    """With the Maxwell-Boltzmann-scaling thermostat each cell's kinetic energy relative to
    its centre of mass, after the collision, is kT times a Gamma(3/2 (n_c - 1)) variate: mapped
    through that CDF it is uniform on [0, 1], pooled over all cells and steps."""
    L = (16, 16, 16)
    kT = 1.7
    p = abi.make_params(L, precision=precision, thermostat=2, kT=kT, seed=41)
    C = int(np.prod(L))
    pits = []
    with abi.Box(p) as box:
        for _ in range(3):
            box.step(1)
            dbg = box.debug_sort()
            r, v = box.state()
            keys = np.empty(box.n, np.int64)
            keys[dbg["ids"]] = dbg["keys"]
            cnt = np.bincount(keys, minlength=C)
            u = np.stack([np.bincount(keys, weights=v[:, d], minlength=C) for d in range(3)], axis=1)
            u /= np.maximum(cnt, 1)[:, None]
            rel = 0.5 * np.bincount(keys, weights=((v - u[keys]) ** 2).sum(axis=1), minlength=C)
            ok = cnt >= 2
            pits.append(stats.gamma.cdf(rel[ok] / kT, 1.5 * (cnt[ok] - 1)))
    assert stats.kstest(np.concatenate(pits), "uniform").pvalue > 1e-3


def test_angular_momentum_conserved_per_cell_mixed():
    """Angular-momentum-conserving collision, mixed form: per cell, momentum and the angular
    momentum about the centre of mass (positions on the shifted grid) are unchanged by the
    collision to FP32 rounding of the stored velocities."""
    L = (12, 10, 8)
    p = mixed_params(L, seed=17, angular=1, dt=0.0)  # dt = 0: the collision alone changes v
    C = int(np.prod(L))
    n = int(round(10 * C))
    r0, v0 = quantize(*inputs.uniform_gaussian_state(L, n, 18), L)
    with abi.Box(p) as box:
        box.set_state(r0, v0, 2)
        abi.mpcd_record_moments(box.h, True)
        box.step(1)
        dbg = box.debug_sort()
        rg, vg = box.state()
        shift = box.moments()[1]
    keys = np.empty(n, np.int64)
    keys[dbg["ids"]] = dbg["keys"]
    # position inside the cell the GPU assigned (periodic images folded next to it)
    cell = np.stack([keys % L[0], (keys // L[0]) % L[1], keys // (L[0] * L[1])], axis=1)
    loc = (rg - shift) / p.a - cell
    loc -= np.array(L) * np.round((loc - 0.5) / np.array(L))
    cnt = np.bincount(keys, minlength=C)
    mean = np.stack([np.bincount(keys, weights=loc[:, d], minlength=C) for d in range(3)], axis=1)
    rho = p.a * (loc - mean[keys] / np.maximum(cnt, 1)[keys, None])
    per = lambda x: np.stack([np.bincount(keys, weights=x[:, d], minlength=C) for d in range(3)], axis=1)
    dLc = per(np.cross(rho, vg)) - per(np.cross(rho, v0))
    scale = np.bincount(keys, weights=np.linalg.norm(rho, axis=1) * np.abs(v0).sum(axis=1), minlength=C) + 1e-30
    assert np.all(np.abs(dLc).max(axis=1) <= 2e-6 * scale)
    dP = per(vg) - per(v0)
    assert np.all(np.abs(dP).max(axis=1) <= 2e-6 * np.bincount(keys, weights=np.abs(v0).sum(axis=1), minlength=C) + 1e-30)
    # the plain collision would change it: the check is not vacuous
    with abi.Box(mixed_params(L, seed=17, dt=0.0)) as box:
        box.set_state(r0, v0, 2)
        box.step(1)
        _, v_plain = box.state()
    assert np.abs(per(np.cross(rho, v_plain)) - per(np.cross(rho, v0))).max() > 1e-3


def test_energy_and_momentum_do_not_drift():
    p = mixed_params((20, 20, 20), seed=13)
    with abi.Box(p) as box:
        r, v = box.state()
        E0 = 0.5 * (v * v).sum()
        box.step(300)
        r, v = box.state()
    assert abs(0.5 * (v * v).sum() / E0 - 1) < 1e-5
    assert np.abs(v.sum(axis=0)).max() < 1e-2
    for d in range(3):
        assert abs(stats.kurtosis(v[:, d], fisher=False) - 3.0) < 0.05


def test_statistics_agree_with_oracle(orc):
    """Shell start (all speeds equal): after 40 steps both forms relax to the same
    velocity moments within sampling noise."""
    L = (16, 16, 16)
    p = mixed_params(L, seed=17)
    n = 40960
    r0, v0 = quantize(*inputs.shell_state(L, n, 17), L)
    with abi.Box(p) as box:
        box.set_state(r0, v0, 0)
        box.step(40)
        _, vg = box.state()
    st = orc.State(r0, v0)
    orc.run(oracle_params(orc, p), st, 40)
    for k in (2, 4):
        mg = np.mean(vg ** k)
        mo = np.mean(st.v ** k)
        assert abs(mg / mo - 1) < (0.002 if k == 2 else 0.03), (k, mg, mo)


def test_runs_are_deterministic():
    """Two runs from the same state give identical bits although the counting atomics hand
    out each cell's members in a different order every time: the per-cell sums are exact."""
    p = mixed_params((12, 12, 12), seed=19)
    outs = []
    for _ in range(2):
        with abi.Box(p) as box:
            box.step(7)
            outs.append(box.state())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_checkpoint_resume_bit_exact():
    """get_state/set_state restarts storage in particle-id order; with order-independent
    cell sums the resumed run still reproduces the uninterrupted one bit for bit."""
    p = mixed_params((10, 10, 10), seed=19)
    with abi.Box(p) as a, abi.Box(p) as b:
        a.step(9)
        b.step(4)
        r, v = b.state()
        b.set_state(r, v, 4)
        b.step(5)
        ra, va = a.state()
        rb, vb = b.state()
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)


def test_crowded_cells_take_the_per_cell_path(orc):
    """Half the particles crowd into a 2x2x2 corner: those warps exceed the staged capacity
    and run cell by cell from global memory; results still match the oracle."""
    L = (8, 8, 8)
    p = mixed_params(L, seed=23, ppc=4.0)
    n = int(round(4 * 512))
    r, v = inputs.uniform_gaussian_state(L, n, 23)
    r[: n // 2] = r[: n // 2] * (2.0 / 8.0)
    r0, v0 = quantize(r, v, L)
    with abi.Box(p) as box:
        box.set_state(r0, v0, 0)
        box.step(1)
        rg, vg = box.state()
    st = orc.State(r0, v0)
    orc.step(oracle_params(orc, p), st)
    rr, vr = st.by_id()
    assert np.abs(vg.sum(axis=0) - v0.sum(axis=0)).max() < 1e-4
    close = np.abs(vg - vr).max(axis=1) <= 5e-6 * np.maximum(np.abs(vr).max(axis=1), 1.0)
    assert close.mean() > 0.99


def test_poiseuille_channel_mixed():
    Lx, Ly, H = 6, 6, 10
    n_bar, g, dt, alpha = 10, 0.01, 0.1, math.radians(130)
    p = mixed_params((Lx, Ly, H), walls_z=1, ppc=n_bar, dt=dt, alpha=alpha, g=(g, 0.0, 0.0), thermostat=1, seed=77)
    f = n_bar * Lx * Ly * H
    nu_kin = dt / 2 * (5 * n_bar / ((n_bar - 1 + math.exp(-n_bar)) * (2 - math.cos(alpha) - math.cos(2 * alpha))) - 1)
    nu_col = (n_bar - 1 + math.exp(-n_bar)) / n_bar * (1 - math.cos(alpha)) / (18 * dt)
    nu = nu_kin + nu_col
    nb = 10
    acc = np.zeros(nb)
    cnt = np.zeros(nb)
    with abi.Box(p) as box:
        assert box.n == f
        box.step(1500)
        for _ in range(100):
            box.step(50)
            r, v = box.state()
            b = np.minimum((r[:, 2] / H * nb).astype(int), nb - 1)
            acc += np.bincount(b, weights=v[:, 0], minlength=nb)
            cnt += np.bincount(b, minlength=nb)
    prof = acc / cnt
    z = (np.arange(nb) + 0.5) * H / nb
    A = np.stack([np.ones(nb), z, z * z], axis=1)
    coef, *_ = np.linalg.lstsq(A, prof, rcond=None)
    nu_fit = -g / (2 * coef[2])
    assert abs(nu_fit / nu - 1) < 0.15, (nu_fit, nu)
    vmax = g * H * H / (8 * nu)
    assert abs(coef[0]) < 0.2 * vmax and abs(-coef[1] / (2 * coef[2]) - H / 2) < 0.05 * H


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_set_state_rejects_invalid_input(precision):
    """Positions outside the box and non-finite velocities are rejected on both entry points,
    naming the first offending particle, and leave the state as it was."""
    import torch
    L = (6, 5, 4)
    p = abi.make_params(L, precision=precision, seed=3)
    with abi.Box(p) as box:
        r0, v0 = box.state()
        for k, (dr, dv) in enumerate([((7, 0), None), ((-1e-9, 2), None), ((float("nan"), 1), None),
                                      (None, (float("inf"), 0)), ((1e300, 2), None)]):
            r, v = r0.copy(), v0.copy()
            i = 11 + k
            if dr:
                r[i, dr[1]] = dr[0] if dr[0] != 7 else 7.0 * L[0]
            if dv:
                v[i, dv[1]] = dv[0]
            with pytest.raises(abi.MpcdError, match="particle %d" % i):
                box.set_state(r, v, 0)
            if torch.cuda.is_available():
                rd = torch.from_numpy(r).cuda()
                vd = torch.from_numpy(v).cuda()
                torch.cuda.synchronize()
                with pytest.raises(abi.MpcdError, match="particle %d" % i):
                    abi.mpcd_set_state_device(box.h, rd, vd, 0)
            r1, v1 = box.state()
            assert np.array_equal(r1, r0) and np.array_equal(v1, v0)


MASS_CASES = [dict(L=(10, 9, 8)), dict(L=(9, 8, 7), g=(0.02, 0.0, 0.01)), dict(L=(10, 9, 8), thermostat=1, kT=1.3),
              dict(L=(11, 9, 8), thermostat=2, kT=1.3), dict(L=(9, 8, 10), walls_z=1, g=(0.02, 0.01, 0.0)),
              dict(L=(8, 9, 12), walls_z=1, g=(0.01, 0.0, 0.0), thermostat=2, ppc=15)]


@pytest.mark.parametrize("case", MASS_CASES, ids=["periodic", "force", "thermostat", "mbs", "walls_force",
                                                   "walls_mbs"])
def test_one_step_with_masses_against_fp64_oracle(orc, case):
    """Per-particle masses in the mixed form (FP32 masses 0.5 to 4 m, mass-weighted exact
    sums): one step from a state and masses both forms represent exactly, against the oracle's
    mass-weighted step, at the mixed form's one-step bounds."""
    from parity import assert_mixed_one_step
    p = mixed_params(seed=15, **case)
    L = tuple(p.L)
    n = int(round(p.ppc * np.prod(L)))
    r0, v0 = quantize(*inputs.uniform_gaussian_state(L, n, 23, a=p.a), L, p.a)
    m = np.random.default_rng(9).uniform(0.5, 4.0, n).astype(np.float32).astype(np.float64) * p.mass
    with abi.Box(p) as box:
        box.set_state(r0, v0, 4)
        box.set_masses(m)
        assert np.array_equal(abi.mpcd_get_masses(box.h), m)
        box.step(1)
        dbg = box.debug_sort()
        rg, vg = box.state()
    st = orc.State(r0, v0, t=4, m=m)
    ref = orc.step(oracle_params(orc, p), st, debug=True)
    rr, vr = st.by_id()
    kg = np.empty(n, np.int64)
    kg[dbg["ids"]] = dbg["keys"]
    ko = np.empty(n, np.int64)
    ko[ref["ids"]] = ref["keys"]
    C = int(np.prod(L)) if not p.walls_z else L[0] * L[1] * (L[2] + 1)
    assert_mixed_one_step(p, kg, ko, rg, vg, rr, vr, ref["shift"], C, what=str(case))


def test_masses_mixed_api_and_conservation():
    """Masses follow their particles through steps and set_state; the mass-weighted momentum
    and kinetic energy are conserved (FP32 rounding); None restores the box mass: the same
    bits as a box that never had masses."""
    p = mixed_params((12, 12, 12), seed=31)
    with abi.Box(p) as box, abi.Box(p) as plain:
        m = np.random.default_rng(8).uniform(0.5, 3.0, box.n).astype(np.float32).astype(np.float64)
        box.set_masses(m)
        r0, v0 = box.state()
        P0, E0 = (m[:, None] * v0).sum(axis=0), 0.5 * (m * (v0 * v0).sum(axis=1)).sum()
        box.step(20)
        r1, v1 = box.state()
        assert np.array_equal(abi.mpcd_get_masses(box.h), m)
        P1, E1 = (m[:, None] * v1).sum(axis=0), 0.5 * (m * (v1 * v1).sum(axis=1)).sum()
        assert np.abs(P1 - P0).max() < 1e-4 * np.abs(m[:, None] * v0).sum() / 3
        assert abs(E1 / E0 - 1) < 1e-5
        box.set_state(r1, v1, 20)
        assert np.array_equal(abi.mpcd_get_masses(box.h), m)
        r0, v0 = plain.state()
        box.set_state(r0, v0, 0)
        box.set_masses(None)
        box.step(3)
        plain.step(3)
        assert np.array_equal(box.state()[1], plain.state()[1])


def test_ensemble_with_masses_equals_boxes_alone():
    boxes = [dict(L=(8, 8, 8), ppc=10, alpha_deg=130, dt=0.1, seed=401),
             dict(L=(12, 10, 8), ppc=6, alpha_deg=95, dt=0.2, seed=402, g=(0.01, 0.0, 0.0))]
    params = [abi.make_params(precision="mixed", thermostat=1, **k) for k in boxes]
    with abi.Box(batch=params) as ens:
        pb, _ = abi.mpcd_box_offsets(ens.h)
        m = np.random.default_rng(5).uniform(0.5, 2.0, ens.n).astype(np.float32).astype(np.float64)
        ens.set_masses(m)
        ens.step(6)
        r, v = ens.state()
    for b, p in enumerate(params):
        with abi.Box(p) as one:
            one.set_masses(m[pb[b]:pb[b + 1]])
            one.step(6)
            r1, v1 = one.state()
        assert np.array_equal(r[pb[b]:pb[b + 1]], r1) and np.array_equal(v[pb[b]:pb[b + 1]], v1), b


@pytest.mark.parametrize("masses", [False, True])
def test_add_momentum_mixed(masses):
    """The coupling hook in the mixed form: the FP32 velocity becomes the FP32 rounding of
    v + dp / m (v and m the stored FP32 values), by particle id."""
    p = mixed_params((9, 8, 7), seed=13)
    with abi.Box(p) as box:
        m = np.random.default_rng(2).uniform(0.5, 3.0, box.n).astype(np.float32).astype(np.float64) if masses else None
        if masses:
            box.set_masses(m)
        box.step(2)
        r0, v0 = box.state()
        dp = np.random.default_rng(3).normal(0.0, 0.1, (box.n, 3))
        abi.mpcd_add_momentum(box.h, dp)
        r1, v1 = box.state()
    mm = (m if masses else np.full(len(v0), p.mass))[:, None]
    assert np.array_equal(r1, r0)
    assert np.array_equal(v1, (v0 + dp / mm).astype(np.float32).astype(np.float64))


def test_add_momentum_ensemble_uses_each_box_mass():
    """In an ensemble without particle masses each particle's increment is divided by its own
    box's mass."""
    params = [abi.make_params((6, 6, 6), precision="mixed", mass=1.0, seed=61),
              abi.make_params((8, 7, 6), precision="mixed", mass=2.5, kT=2.5, seed=62)]
    with abi.Box(batch=params) as ens:
        pb, _ = abi.mpcd_box_offsets(ens.h)
        ens.step(2)
        r0, v0 = ens.state()
        dp = np.random.default_rng(4).normal(0.0, 0.2, (ens.n, 3))
        abi.mpcd_add_momentum(ens.h, dp)
        r1, v1 = ens.state()
    m = np.empty((len(v0), 1))
    m[pb[0]:pb[1]] = 1.0
    m[pb[1]:pb[2]] = 2.5
    assert np.array_equal(r1, r0)
    assert np.array_equal(v1, (v0 + dp / m).astype(np.float32).astype(np.float64))
