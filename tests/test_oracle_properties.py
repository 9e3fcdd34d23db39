"""Property pins for the oracle over random small boxes and parameters (hypothesis).

For any box, cell size, angle, time step and seed, one oracle step must:
  * put every particle in a valid cell, with counts summing to N and offsets their prefix
    sum, and a perm that is the stable argsort of the keys;
  * keep every cell's momentum and kinetic energy (plain collision), or its momentum and
    angular momentum about the centre of mass (angular-momentum conservation), with or
    without per-particle masses;
  * leave positions inside the periodic box.
These hold whatever the arithmetic in between, so they catch slips that the fixed cases of
the other pin files could miss for some geometry.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

from paper_2212_11878_gb300 import inputs  # noqa: E402

boxes = st.tuples(st.integers(1, 5), st.integers(1, 5), st.integers(1, 5))
params = st.fixed_dictionaries({
    "a": st.sampled_from([1.0, 0.5, 0.7, 1.3]),
    "alpha_deg": st.floats(5.0, 175.0),
    "dt": st.sampled_from([0.0, 0.05, 0.1, 0.37]),
    "ppc": st.sampled_from([1.5, 4.0, 10.0]),
    "seed": st.integers(0, 2 ** 40),
})


def _per_cell(keys, C, x):
    return np.stack([np.bincount(keys, weights=x[:, d], minlength=C) for d in range(3)], axis=1)


def _run(orc, L, kw, angular, masses, state_seed):
    p = orc.make_params(L, angular=angular, **kw)
    n = max(1, int(round(p.ppc * np.prod(L))))
    r, v = inputs.uniform_gaussian_state(L, n, state_seed, a=p.a)
    m = inputs.particle_masses(n, state_seed, 0.5, 3.0) if masses else None
    st_ = orc.State(r, v, m=m)
    out = orc.step(p, st_, debug=True)
    return p, n, r, v, m, st_, out


@settings(max_examples=40, deadline=None)
@given(L=boxes, kw=params, angular=st.booleans(), masses=st.booleans(), state_seed=st.integers(0, 10 ** 6))
def test_step_invariants(orc, L, kw, angular, masses, state_seed):
    p, n, r0, v0, m, s1, out = _run(orc, L, kw, int(angular), masses, state_seed)
    C = orc.num_cells(p)
    keys, counts, offsets, perm = out["keys"], out["counts"], out["offsets"], out["perm"]
    # the sort
    assert keys.min() >= 0 and keys.max() < C
    assert np.array_equal(counts, np.bincount(keys, minlength=C)) and counts.sum() == n
    assert offsets[0] == 0 and np.array_equal(offsets[1:], np.cumsum(counts))
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))
    # positions stay in the periodic box
    box = np.array(L, float) * p.a
    assert np.all(s1.r >= 0) and np.all(s1.r < box)
    # per-cell conservation (no force: streaming leaves v alone, so v0 is the pre-collision v)
    w = np.ones(n) if m is None else m
    scale = np.bincount(keys, weights=w * np.abs(v0).sum(axis=1), minlength=C) + 1e-300
    dP = _per_cell(keys, C, w[:, None] * s1.v) - _per_cell(keys, C, w[:, None] * v0)
    assert np.all(np.abs(dP).max(axis=1) <= 1e-12 * scale)
    if not angular:
        E0 = np.bincount(keys, weights=w * (v0 * v0).sum(axis=1), minlength=C)
        E1 = np.bincount(keys, weights=w * (s1.v * s1.v).sum(axis=1), minlength=C)
        assert np.all(np.abs(E1 - E0) <= 1e-12 * np.maximum(E0, 1e-300))
    else:
        q = (s1.r - out["shift"]) / p.a
        loc = q - np.floor(q)
        M = np.bincount(keys, weights=w, minlength=C)
        com = _per_cell(keys, C, w[:, None] * loc) / np.maximum(M, 1e-300)[:, None]
        rho = p.a * (loc - com[keys])
        dL = _per_cell(keys, C, w[:, None] * np.cross(rho, s1.v)) - _per_cell(keys, C, w[:, None] * np.cross(rho, v0))
        lscale = np.bincount(keys, weights=w * np.linalg.norm(rho, axis=1) * np.abs(v0).sum(axis=1), minlength=C)
        # collinear cells of three or more are left uncorrected (a singular inertia tensor)
        cnt = counts
        ok = np.ones(C, bool)
        for c in np.nonzero(cnt >= 3)[0]:
            rr = rho[keys == c]
            I = ((w[keys == c] * (rr * rr).sum(axis=1)).sum() * np.eye(3)
                 - (w[keys == c][:, None] * rr).T @ rr)
            ev = np.linalg.eigvalsh(I)
            ok[c] = ev[0] > 1e-8 * max(ev[-1], 1e-300)
        assert np.all(np.abs(dL).max(axis=1)[ok] <= 1e-11 * (lscale[ok] + 1e-300))
