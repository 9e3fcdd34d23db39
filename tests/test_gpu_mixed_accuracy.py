"""Error of the mixed-precision form against the FP64 oracle and the FP64 GPU form, per
quantity, on a 64^3 box (2,621,440 particles) and a small Poiseuille channel.

Each test asserts a bound on its quantity.  If the environment names a file in
MPCD_ACCURACY_REPORT, each test also adds its measured errors to that JSON file.
  * one step from a state both forms represent exactly: position and velocity errors
    against the oracle, and how many cell keys differ (each lies within FP32 rounding of a
    shifted face);
  * per collision and per cell: momentum and kinetic energy after the collision against
    the exact sums before it;
  * 500 steps from the same start in both forms: <v^2> drift and the normalised fourth
    moment <v^4>/<v^2>^2 (Maxwell-Boltzmann: 5/3), mixed against FP64;
  * Poiseuille flow between walls: the time-averaged profile of each form, the two against
    each other and against the parabola with the SRD viscosity.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2212_11878_gb300 import abi, inputs
from parity import oracle_params, periodic_diff
from test_gpu_mixed import quantize

pytestmark = pytest.mark.gpu

L64 = (64, 64, 64)


def report(section, values):
    path = os.environ.get("MPCD_ACCURACY_REPORT")
    if not path:
        return
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[section] = values
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)


def test_one_step_error_against_oracle_64(orc):
    p = abi.make_params(L64, precision="mixed", seed=21)
    n = int(round(p.ppc * np.prod(L64)))
    r0, v0 = quantize(*inputs.uniform_gaussian_state(L64, n, 64), L64)
    with abi.Box(p) as box:
        box.set_state(r0, v0, 7)
        box.step(1)
        dbg = box.debug_sort()
        rg, vg = box.state()
    st = orc.State(r0, v0, t=7)
    ref = orc.step(oracle_params(orc, p), st, debug=True)
    rr, vr = st.by_id()
    kg = np.empty(n, np.int64)
    kg[dbg["ids"]] = dbg["keys"]
    ko = np.empty(n, np.int64)
    ko[ref["ids"]] = ref["keys"]
    bad = kg != ko
    C = int(np.prod(L64))
    clean = np.isin(ko, np.setdiff1d(np.arange(C), np.concatenate([kg[bad], ko[bad]])))
    dr = periodic_diff(rg, rr, np.array(L64, float)).max(axis=1)
    dv = np.abs(vg - vr).max(axis=1)[clean]
    sig = math.sqrt(p.kT / p.mass)
    rel_v = dv / np.maximum(np.abs(vr).max(axis=1)[clean], sig)
    out = {"particles": n, "key_disagreements": int(bad.sum()), "key_disagreement_fraction": float(bad.mean()),
           "position_abs_max": float(dr.max()), "position_abs_rms": float(np.sqrt((dr ** 2).mean())),
           "velocity_rel_max": float(rel_v.max()), "velocity_rel_rms": float(np.sqrt((rel_v ** 2).mean())),
           "velocity_cells_compared": float(clean.mean())}
    report("one_step_vs_oracle_64", out)
    assert out["key_disagreement_fraction"] <= 2e-5
    assert out["position_abs_max"] <= 64 * 2 ** -23
    assert out["velocity_rel_max"] <= 5e-6


def test_per_cell_conservation_per_collision_64():
    p = abi.make_params(L64, precision="mixed", seed=22)
    C = int(np.prod(L64))
    worst_p, worst_e, rms_e = [], [], []
    with abi.Box(p) as box:
        box.step(20)
        abi.mpcd_record_moments(box.h, True)
        for _ in range(3):
            box.step(1)
            mom, _ = box.moments()
            dbg = box.debug_sort()
            rg, vg = box.state()
            keys = np.empty(box.n, np.int64)
            keys[dbg["ids"]] = dbg["keys"]
            P = np.stack([np.bincount(keys, weights=vg[:, d], minlength=C) for d in range(3)], axis=1)
            E = 0.5 * np.bincount(keys, weights=(vg * vg).sum(axis=1), minlength=C)
            scale = np.bincount(keys, weights=np.abs(vg).sum(axis=1), minlength=C) + 1e-30
            occ = mom[:, 0] >= 2
            dp = np.abs(P - mom[:, 1:4]).max(axis=1)[occ] / scale[occ]
            de = np.abs(E - mom[:, 4])[occ] / mom[occ, 4]
            worst_p.append(float(dp.max()))
            worst_e.append(float(de.max()))
            rms_e.append(float(np.sqrt((de ** 2).mean())))
    out = {"cells": C, "momentum_rel_max": max(worst_p), "energy_rel_max": max(worst_e),
           "energy_rel_rms": max(rms_e), "note": "relative to the cell's sum of |v| (momentum) or kinetic energy"}
    report("per_cell_conservation_64", out)
    assert out["momentum_rel_max"] <= 2e-6
    assert out["energy_rel_max"] <= 2e-6


def moments(v):
    v2 = (v * v).sum(axis=1)
    return v2.mean(), (v2 * v2).mean() / v2.mean() ** 2


def test_velocity_moments_500_steps_mixed_vs_fp64():
    n = int(round(10 * np.prod(L64)))
    r0, v0 = quantize(*inputs.uniform_gaussian_state(L64, n, 65), L64)
    res = {}
    for prec in ("fp64", "mixed"):
        p = abi.make_params(L64, precision=prec, seed=23)
        with abi.Box(p) as box:
            box.set_state(r0, v0, 0)
            m2_0, _ = moments(box.state()[1])
            box.step(500)
            m2, q = moments(box.state()[1])
        res[prec] = {"v2_drift_rel": float(m2 / m2_0 - 1), "v4_over_v2sq": float(q)}
    res["v4_over_v2sq_mixed_minus_fp64"] = res["mixed"]["v4_over_v2sq"] - res["fp64"]["v4_over_v2sq"]
    res["maxwell_v4_over_v2sq"] = 5.0 / 3.0
    report("moments_500_steps_64", res)
    assert abs(res["fp64"]["v2_drift_rel"]) < 1e-10
    assert abs(res["mixed"]["v2_drift_rel"]) < 1e-5
    # both forms relax to the same distribution; sampling noise of the ratio ~ 3e-3
    assert abs(res["v4_over_v2sq_mixed_minus_fp64"]) < 0.01
    assert abs(res["mixed"]["v4_over_v2sq"] - 5 / 3) < 0.01


def test_poiseuille_profile_mixed_vs_fp64():
    Lx, Ly, H = 8, 8, 16
    n_bar, g, dt, alpha = 10, 0.01, 0.1, math.radians(130)
    nu_kin = dt / 2 * (5 * n_bar / ((n_bar - 1 + math.exp(-n_bar)) * (2 - math.cos(alpha) - math.cos(2 * alpha))) - 1)
    nu_col = (n_bar - 1 + math.exp(-n_bar)) / n_bar * (1 - math.cos(alpha)) / (18 * dt)
    nu = nu_kin + nu_col
    vmax = g * H * H / (8 * nu)
    nb = 16
    z = (np.arange(nb) + 0.5) * H / nb
    profiles = {}
    for prec in ("fp64", "mixed"):
        p = abi.make_params((Lx, Ly, H), precision=prec, walls_z=1, ppc=n_bar, dt=dt, alpha=alpha, g=(g, 0.0, 0.0),
                            thermostat=1, seed=78)
        acc = np.zeros(nb)
        cnt = np.zeros(nb)
        with abi.Box(p) as box:
            box.step(2000)
            for _ in range(200):
                box.step(20)
                r, v = box.state()
                b = np.minimum((r[:, 2] / H * nb).astype(int), nb - 1)
                acc += np.bincount(b, weights=v[:, 0], minlength=nb)
                cnt += np.bincount(b, minlength=nb)
        profiles[prec] = acc / cnt
    theory = g / (2 * nu) * z * (H - z)
    out = {"vmax_theory": vmax,
           "mixed_vs_fp64_rms_over_vmax": float(np.sqrt(((profiles["mixed"] - profiles["fp64"]) ** 2).mean()) / vmax)}
    for prec in ("fp64", "mixed"):
        A = np.stack([np.ones(nb), z, z * z], axis=1)
        coef, *_ = np.linalg.lstsq(A, profiles[prec], rcond=None)
        out[prec] = {"nu_fit_over_theory": float(-g / (2 * coef[2]) / nu),
                     "rms_vs_parabola_over_vmax": float(np.sqrt(((profiles[prec] - theory) ** 2).mean()) / vmax)}
    report("poiseuille_8x8x16", out)
    assert out["mixed_vs_fp64_rms_over_vmax"] < 0.05
    for prec in ("fp64", "mixed"):
        assert abs(out[prec]["nu_fit_over_theory"] - 1) < 0.15
