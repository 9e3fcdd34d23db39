"""GPU parity of the FP64 SRD step (libmpcd through the C ABI) against the FP64 CPU oracle,
from identical states: keys, counts, offsets, perm bit-exact; positions and velocities
within 1e-12 relative (tests/parity.py states the bound)."""
import math

import numpy as np
import pytest

from paper_2212_11878_gb300 import abi, inputs
from parity import assert_sort_equal, assert_state_close, oracle_params

pytestmark = pytest.mark.gpu


def angular_multiplier(p, rr, ref, m=None):
    """Per-particle (id order) factor on the 1e-12 bound of one step of the angular-momentum-
    conserving collision from identical states.  Its correction omega = I^-1 dL turns rounding
    differences of the rotated velocities (a few ulps: the two sides round the rotation
    differently) into velocity differences about cond(I) ulps large, cond(I) the condition
    number of the cell's inertia tensor; nearly collinear cells of three particles make it
    large.  The factor is max(1, cond(I)/100) (1e-12 / 100 = 1e-14, about 50 ulps) of this
    step's cell only: the multi-step runs restart both sides from the oracle's state every
    step, so no factor is carried forward.  test_angular_correction_decomposed holds the part
    of the velocity before the correction to the flat 1e-12."""
    n = len(rr)
    keys = np.empty(n, np.int64)
    keys[ref["ids"]] = ref["keys"]
    q = (rr - ref["shift"]) / p.a
    loc = q - np.floor(q)
    mult = np.ones(n)
    order = np.argsort(keys, kind="stable")
    bounds = np.searchsorted(keys[order], np.arange(keys.max() + 2))
    for c in range(len(bounds) - 1):
        idx = order[bounds[c]:bounds[c + 1]]
        if len(idx) < 2:
            continue
        w = np.ones(len(idx)) if m is None else m[idx]
        rho = loc[idx] - (w[:, None] * loc[idx]).sum(axis=0) / w.sum()
        I = (w * (rho * rho).sum(axis=1)).sum() * np.eye(3) - (w[:, None] * rho).T @ rho
        ev = np.linalg.eigvalsh(I)
        cond = ev[-1] / max(ev[0], ev[-1] * 1e-16) if len(idx) > 2 else ev[-1] / max(ev[1], ev[-1] * 1e-16)
        mult[idx] = max(1.0, cond / 100.0)
    return mult


def run_pair(orc, p, r, v, steps, t0=0, check_sort_every=True, masses=None, displacement_scale=False):
    """Advance the library and the oracle from the same state (and per-particle masses, in
    particle-id order); compare after every step."""
    box = abi.Box(p)
    try:
        box.set_state(r, v, t0)
        if masses is not None:
            box.set_masses(masses)
        op = oracle_params(orc, p)
        st = orc.presort(op, orc.State(r, v, t=t0, m=masses))  # set_state stores in cell order
        mult = np.ones(len(r))
        for k in range(steps):
            box.step(1)
            ref = orc.step(op, st, debug=check_sort_every or bool(p.angular))
            if check_sort_every:
                assert_sort_equal(box.debug_sort(), ref)
            rg, vg = box.state()
            rr, vr = st.by_id()
            if p.angular:
                mult = angular_multiplier(p, rr, ref, masses)
            r_scale = np.abs(vr).max(axis=1) * p.dt if displacement_scale else None
            assert_state_close(rg, vg, rr, vr, p, tol=1e-12 * mult, what="step %d" % (t0 + k + 1), r_scale=r_scale)
            if p.angular:  # restart both sides from the oracle's state: one-step comparisons
                box.set_state(rr, vr, st.t)
                st = orc.presort(op, orc.State(rr, vr, t=st.t, m=masses))
        return box.state(), st
    finally:
        box.close()


CASES = {
    "cubic_L16": dict(L=(16, 16, 16)),
    "ragged_5x7x3": dict(L=(5, 7, 3)),
    "single_cell": dict(L=(1, 1, 1), ppc=12),
    "sparse": dict(L=(9, 8, 7), ppc=0.7),
    "dense": dict(L=(4, 4, 4), ppc=40),
    "a_half": dict(L=(6, 6, 6), a=0.5),
    "a_non_pow2": dict(L=(6, 5, 4), a=0.7),
    "mass_dt": dict(L=(6, 6, 6), mass=1.7, dt=0.37, kT=2.5, alpha_deg=77.0),
    "no_resort": dict(L=(8, 8, 8), resort_k=0),
    "resort_3": dict(L=(8, 8, 8), resort_k=3),
    "dense_resort_1": dict(L=(4, 4, 4), ppc=40, resort_k=1),     # cells above 16 members re-sorted
    "sparse_resort_1": dict(L=(9, 8, 7), ppc=3, resort_k=1),     # every cell through the network
    "force": dict(L=(6, 6, 6), g=(0.01, -0.02, 0.005)),
    "walls": dict(L=(6, 5, 8), walls_z=1, g=(0.01, 0.0, 0.0)),
    "walls_thermo": dict(L=(6, 5, 8), walls_z=1, g=(0.02, 0.0, 0.0), thermostat=1, ppc=15),
    "thermo_periodic": dict(L=(6, 6, 6), thermostat=1, kT=0.8),
    "mbs_periodic": dict(L=(7, 6, 6), thermostat=2, kT=0.8),
    "walls_mbs": dict(L=(6, 5, 8), walls_z=1, g=(0.02, 0.0, 0.0), thermostat=2, ppc=15),
    "mbs_sparse": dict(L=(8, 8, 8), thermostat=2, ppc=2.5),
    "angular": dict(L=(7, 6, 5), angular=1),
    "angular_mbs": dict(L=(6, 6, 6), angular=1, thermostat=2, kT=0.9),
    "angular_resort_force": dict(L=(8, 7, 6), angular=1, resort_k=3, g=(0.01, 0.0, -0.02)),
    "angular_sparse_a_half": dict(L=(8, 8, 8), angular=1, ppc=2.5, a=0.5),
}


@pytest.mark.parametrize("name", list(CASES))
def test_steps_match_oracle(orc, name):
    kw = dict(CASES[name])
    p = abi.make_params(seed=1000 + len(name), **kw)
    n = int(round(p.ppc * p.L[0] * p.L[1] * p.L[2]))
    r, v = inputs.uniform_gaussian_state(tuple(p.L), n, 31 + len(name), a=p.a, kT=p.kT, mass=p.mass)
    run_pair(orc, p, r, v, steps=6, t0=3)


MASS_CASES = {
    "masses": dict(L=(7, 6, 5)),
    "masses_walls_thermostat": dict(L=(6, 5, 8), walls_z=1, g=(0.01, 0.0, 0.0), thermostat=1, ppc=12),
    "masses_mbs_resort": dict(L=(6, 6, 6), thermostat=2, resort_k=2),
    "masses_angular": dict(L=(6, 6, 5), angular=1),
    "masses_angular_sparse": dict(L=(7, 7, 7), angular=1, ppc=3, resort_k=3),
}


@pytest.mark.parametrize("name", list(MASS_CASES))
def test_particle_masses_match_oracle(orc, name):
    """Per-particle masses (Listing 4's m), 0.5 to 4 times the box mass, against the oracle
    with the same masses; keys and sort bit-exact, state within the FP64 bound."""
    p = abi.make_params(seed=2000 + len(name), **MASS_CASES[name])
    n = int(round(p.ppc * p.L[0] * p.L[1] * p.L[2]))
    r, v = inputs.uniform_gaussian_state(tuple(p.L), n, 41 + len(name), a=p.a)
    m = np.random.default_rng(len(name)).uniform(0.5, 4.0, n) * p.mass
    run_pair(orc, p, r, v, steps=6, t0=2, masses=m)


def test_particle_masses_api():
    p = abi.make_params((8, 8, 8), seed=5, resort_k=2)
    n = int(round(p.ppc * 512))
    m = np.random.default_rng(1).uniform(0.5, 3.0, n)
    with abi.Box(p) as box, abi.Box(p) as plain:
        assert np.array_equal(abi.mpcd_get_masses(box.h), np.full(n, p.mass))
        box.set_masses(m)
        box.step(5)  # two re-sorts
        assert np.array_equal(abi.mpcd_get_masses(box.h), m)
        r, v = box.state()
        box.set_state(r, v, 5)  # storage rebuilt from id order: masses follow
        assert np.array_equal(abi.mpcd_get_masses(box.h), m)
        # the box mass restored: the same steps as a box that never had masses
        r0, v0 = plain.state()
        box.set_state(r0, v0, 0)
        box.set_masses(None)
        box.step(3)
        plain.step(3)
        assert np.array_equal(box.state()[1], plain.state()[1])
        for bad in (np.full(n, -1.0), np.full(n, np.nan), np.ones(n - 1)):
            with pytest.raises((abi.MpcdError, ValueError)):
                box.set_masses(bad)
    with abi.Box(abi.make_params((4, 4, 4), precision="mixed", angular=1)) as mixed:
        with pytest.raises(abi.MpcdError) as ei:  # masses with angular conservation: FP64 form only
            mixed.set_masses(np.ones(mixed.n))
        assert ei.value.code == abi.MPCD_ERR_ARG


def test_face_positions_bit_exact_keys(orc):
    p = abi.make_params((6, 6, 6), dt=0.0, ppc=2000 / 216)
    r, v = inputs.face_state((6, 6, 6), 2000, 5)
    run_pair(orc, p, r, v, steps=3)


@pytest.mark.parametrize("kw", [dict(), dict(a=0.5), dict(a=2.0), dict(walls_z=1)],
                         ids=["a1", "a_half", "a2", "walls"])
def test_keys_within_ulps_of_shifted_faces(orc, kw):
    """Coordinates a few ulps either side of the faces of the grids that the next three steps
    shift to (dt = 0: nothing moves), the rest uniform: each cell key is the floor of the
    rounded FP64 difference (r - s) / a bit for bit, however the kernel reaches it (in fixed
    point away from a face, by the FP64 subtraction next to one).  One step per call (the
    streaming kernel) and three in one call (the fused rotate-and-stream pass after the
    first)."""
    L = (6, 5, 7)
    p = abi.make_params(L, dt=0.0, seed=303, **kw)
    op = oracle_params(orc, p)
    a = p.a
    box_len = np.asarray(L, dtype=np.float64) * a
    n = int(round(p.ppc * np.prod(L)))
    rng = np.random.default_rng(17)
    r = rng.uniform(0.0, 1.0, (n, 3)) * box_len
    per_step = n // 4
    for j in range(3 * per_step):
        s = orc.shift(op, j // per_step + 1)
        for d in range(3):
            while True:
                x = s[d] + int(rng.integers(0, L[d] + 1)) * a
                k = int(rng.integers(-6, 7))
                for _ in range(abs(k)):
                    x = np.nextafter(x, np.inf if k > 0 else -np.inf)
                if 0.0 <= x < box_len[d]:
                    break
            r[j, d] = x
    v = rng.standard_normal((n, 3))
    run_pair(orc, p, r, v, steps=3)
    with abi.Box(p) as box:
        box.set_state(r, v, 0)
        box.step(3)
        st = orc.presort(op, orc.State(r, v, t=0))
        for t in range(1, 4):
            ref = orc.step(op, st, debug=True)
            assert np.array_equal(ref["shift"], orc.shift(op, t))
        assert_sort_equal(box.debug_sort(), ref)
        rg, vg = box.state()
        rr, vr = st.by_id()
        assert_state_close(rg, vg, rr, vr, p, tol=1e-12, what="three steps in one call")


def test_empty_box(orc):
    p = abi.make_params((4, 4, 4), ppc=0.0)
    with abi.Box(p) as box:
        assert box.n == 0
        box.step(3)
        dbg = box.debug_sort()
        assert np.all(dbg["counts"] == 0) and np.all(dbg["offsets"] == 0)


def test_init_matches_oracle(orc):
    w = inputs.WORKLOADS["fp64_L16"]
    p = abi.params_from_workload(w)
    with abi.Box(p) as box:
        rg, vg = box.state()
    rr, vr = orc.init(oracle_params(orc, p), box_n := rg.shape[0])
    assert box_n == w.n_particles
    assert np.array_equal(rg, rr)                 # U53 * L: exact on both sides
    assert_state_close(rg, vg, rr, vr, p, what="init")
    assert np.abs(vg.sum(axis=0)).max() < 1e-10


def test_trajectory_100_steps_L16(orc):
    """The small workload: 16^3 cells, 40,960 particles, 100 steps, compared by particle id
    after every 10 steps and in full at the end."""
    w = inputs.WORKLOADS["fp64_L16"]
    p = abi.params_from_workload(w)
    op = oracle_params(orc, p)
    r0, v0 = orc.init(op, w.n_particles)
    st = orc.presort(op, orc.State(r0, v0))
    with abi.Box(p) as box:
        box.set_state(r0, v0, 0)
        for _ in range(10):
            box.step(10)
            orc.run(op, st, 10)
            rg, vg = box.state()
            rr, vr = st.by_id()
            assert_state_close(rg, vg, rr, vr, p, what="t=%d" % st.t)
        box.step(1)
        ref = orc.step(op, st, debug=True)
        assert_sort_equal(box.debug_sort(), ref)


def test_moments_match_oracle(orc):
    p = abi.make_params((7, 6, 5), mass=1.3)
    n = int(round(p.ppc * 7 * 6 * 5))
    r, v = inputs.uniform_gaussian_state((7, 6, 5), n, 8)
    with abi.Box(p) as box:
        box.set_state(r, v, 0)
        abi.mpcd_record_moments(box.h, True)
        box.step(1)
        mom, shift = box.moments()
    op = oracle_params(orc, p)
    st = orc.presort(op, orc.State(r, v))
    ref = orc.step(op, st, debug=True)
    assert np.array_equal(shift, ref["shift"])
    assert np.array_equal(mom[:, 0], ref["moments"][:, 0]) or np.allclose(mom[:, 0], ref["moments"][:, 0], rtol=1e-15)
    scale = np.maximum(np.abs(ref["moments"]).max(axis=0), 1.0)
    assert np.all(np.abs(mom - ref["moments"]) <= 1e-12 * scale)


def test_graph_and_timed_paths_agree():
    """Graph replay and the event-timed launch path run the same kernels: identical bits."""
    p = abi.make_params((12, 12, 12), resort_k=2)
    outs = []
    for timed in (False, True):
        with abi.Box(p) as box:
            if timed:
                abi.mpcd_timing(box.h, True)
            box.step(7)
            outs.append(box.state())
            if timed:
                t = abi.mpcd_timing_read(box.h)
                # one mpcd_step(7) call: the first step streams alone, the next six fuse the
                # previous rotation with their streaming, and the last rotation runs alone
                assert t["collide"][1] == 7 and t["scan"][1] == 21
                assert t["stream_bin"][1] == 1 and t["rotate_stream"][1] == 6 and t["rotate"][1] == 1
                assert all(ms >= 0 for ms, _ in t.values())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("resort_k", [0, 3])
def test_checkpoint_resume_bit_exact(resort_k):
    """Run 2n steps, or n steps + get_state/set_state + n steps: identical bits.  The cell
    sums are exact (order-independent), so this holds even when the restored run keeps its
    particles in a different storage order than the uninterrupted one."""
    p = abi.make_params((10, 10, 10), resort_k=resort_k)
    with abi.Box(p) as a, abi.Box(p) as b:
        a.step(8)
        b.step(4)
        r, v = b.state()
        b.set_state(r, v, 4)
        b.step(4)
        ra, va = a.state()
        rb, vb = b.state()
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)


def test_dense_pair_at_two_densities(orc):
    """The dense FP64 pair (cell_frame + rotate) at 16 and at 10 particles per cell: keys and
    perm bit-exact, state within tolerance.  (The per-cell FP64 kernel on a plain periodic box
    is compared with this pair by tests/test_zz_no_alloc.py, whose entry point runs it.)"""
    for ppc in (16.0, 10.0):
        p = abi.make_params((8, 8, 8), ppc=ppc, seed=77)
        n = int(round(ppc * 512))
        r, v = inputs.uniform_gaussian_state((8, 8, 8), n, 78)
        run_pair(orc, p, r, v, steps=3)


def test_conservation_on_gpu():
    p = abi.make_params((20, 20, 20))
    with abi.Box(p) as box:
        r, v = box.state()
        P0, E0 = v.sum(axis=0), 0.5 * (v * v).sum()
        box.step(50)
        r, v = box.state()
    assert np.abs(v.sum(axis=0) - P0).max() < 1e-9
    assert abs(0.5 * (v * v).sum() / E0 - 1) < 1e-12


def test_errors_reported():
    p = abi.make_params((4, 4, 4))
    with abi.Box(p) as box:
        with pytest.raises(abi.MpcdError) as e:
            box.debug_sort()
        assert e.value.code == abi.MPCD_ERR_STATE
        with pytest.raises(abi.MpcdError) as e:
            box.moments()
        assert e.value.code == abi.MPCD_ERR_STATE
        r, v = box.state()
        r[3, 1] = 4.0                              # outside [0, L a)
        with pytest.raises(abi.MpcdError) as e:
            box.set_state(r, v)
        assert e.value.code == abi.MPCD_ERR_ARG
        rc = abi.lib().mpcd_set_state(box.h, box.n - 1, r.ctypes.data, v.ctypes.data, 0)
        assert rc == abi.MPCD_ERR_ARG
        # the handle is still usable after argument errors
        box.step(2)
        assert abi.mpcd_steps_done(box.h) == 2
        assert abi.mpcd_launch_count(box.h) > 0


ANGULAR_CASES = {
    "angular": (dict(L=(7, 6, 5)), False),
    "angular_mbs": (dict(L=(6, 6, 6), thermostat=2, kT=0.9), False),
    "angular_sparse_a_half": (dict(L=(8, 8, 8), ppc=2.5, a=0.5), False),
    "angular_masses": (dict(L=(6, 6, 5)), True),
}


@pytest.mark.parametrize("name", list(ANGULAR_CASES))
def test_angular_correction_decomposed(orc, name):
    """One step of the angular-momentum-conserving collision split into its two parts, each
    against the oracle from identical states:
      - the velocity before the correction (the same boxes with angular = 0) to the flat 1e-12
        bound, with no condition-number factor;
      - the correction omega x rho_i itself (angular = 1 minus angular = 0, per particle) to
        1e-12 max(|v|, sqrt(kT/m)) times max(1, cond(I)/100) of the particle's cell, the only
        place where the inertia tensor's conditioning enters.
    The full velocities then agree within the sum of the two bounds."""
    kw, with_masses = ANGULAR_CASES[name]
    base = abi.make_params(seed=3000 + len(name), resort_k=0, **kw)
    n = int(round(base.ppc * base.L[0] * base.L[1] * base.L[2]))
    r, v = inputs.uniform_gaussian_state(tuple(base.L), n, 61 + len(name), a=base.a, kT=base.kT)
    m = np.random.default_rng(len(name)).uniform(0.5, 4.0, n) if with_masses else None
    t0 = 6
    out = {}
    for ang in (0, 1):
        p = abi.make_params(seed=3000 + len(name), resort_k=0, angular=ang, **kw)
        op = oracle_params(orc, p)
        with abi.Box(p) as box:
            box.set_state(r, v, t0)
            if m is not None:
                box.set_masses(m)
            box.step(1)
            rg, vg = box.state()
        st = orc.presort(op, orc.State(r, v, t=t0, m=m))
        ref = orc.step(op, st, debug=True)
        rr, vr = st.by_id()
        out[ang] = (p, rg, vg, rr, vr, ref)
    p0, rg0, vg0, rr0, vr0, _ = out[0]
    p1, rg1, vg1, rr1, vr1, ref1 = out[1]
    assert_state_close(rg0, vg0, rr0, vr0, p0, what="before the correction")   # flat 1e-12
    assert np.array_equal(rr0, rr1) and np.array_equal(rg0, rg1)
    mult = angular_multiplier(p1, rr1, ref1, m)
    scale = np.maximum(np.abs(vr1).max(axis=1), math.sqrt(p1.kT / p1.mass))
    corr_gpu = vg1 - vg0
    corr_orc = vr1 - vr0
    assert np.abs(corr_orc).max() > 1e-3                                        # the correction is real
    err = np.abs(corr_gpu - corr_orc).max(axis=1)
    bound = 1e-12 * scale * (2.0 + mult)   # the two flat parts plus the conditioned correction
    assert (err <= bound).all(), (err / bound).max()


def test_fast_particles_fallback_sums_in_storage_order(orc):
    """A velocity component of 2^16 or more is beyond the exact fixed-point sums; such a
    cell is summed in plain FP64 with its members in storage order, the oracle's order, so
    the result matches the oracle and repeats bit for bit although the counting atomics
    hand out the slots in a different order on every run.  No re-sort (k = 0): the cells'
    entries arrive in atomic order every step.  A fast particle crosses the box about a
    thousand times per step, so its position bound scales with its displacement |v| dt."""
    p = abi.make_params((6, 6, 6), seed=71, resort_k=0)
    n = int(round(p.ppc * 216))
    r, v = inputs.uniform_gaussian_state((6, 6, 6), n, 72)
    v[::97, 0] = 7.0e4 * np.where(np.arange(0, n, 97) % 2 == 0, 1.0, -1.0)   # > 2^16
    outs = [run_pair(orc, p, r, v, steps=4, displacement_scale=True)[0] for _ in range(2)]
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("kw", [dict(), dict(angular=1), dict(masses=True), dict(g=(0.01, 0.0, -0.02), a=0.7)],
                         ids=["plain", "angular", "masses", "force_a_non_pow2"])
def test_fused_and_separate_passes_identical(kw):
    """The tuning's fuse switch only changes how the rotation is scheduled (in the next step's
    streaming pass, or in a pass of its own): identical bits, across re-sorts and across
    several mpcd_step calls."""
    kw = dict(kw)
    masses = kw.pop("masses", False)
    p = abi.make_params((10, 9, 8), resort_k=3, seed=91, **kw)
    outs = []
    for fuse in (1, 0):
        with abi.Box(p) as box:
            abi.mpcd_set_tuning(box.h, fuse=fuse)
            if masses:
                box.set_masses(np.random.default_rng(4).uniform(0.5, 3.0, box.n))
            for n in (1, 3, 4, 2):
                box.step(n)
            outs.append(box.state())
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("masses", [False, True])
def test_add_momentum_fp64_exact(masses):
    """The coupling hook: v_i + dp_i / m_i, each operation rounded once (numpy's IEEE
    arithmetic gives the same bits), by particle id whatever the storage order; the host and
    the device entry points agree."""
    torch = pytest.importorskip("torch")
    p = abi.make_params((8, 7, 6), seed=5, resort_k=2)
    with abi.Box(p) as box:
        m = np.random.default_rng(2).uniform(0.5, 3.0, box.n) if masses else None
        if masses:
            box.set_masses(m)
        box.step(3)  # storage re-sorted
        r0, v0 = box.state()
        dp = np.random.default_rng(3).normal(0.0, 0.1, (box.n, 3))
        abi.mpcd_add_momentum(box.h, dp)
        r1, v1 = box.state()
        mm = (m if masses else np.full(box.n, p.mass))[:, None]
        assert np.array_equal(r1, r0) and np.array_equal(v1, v0 + dp / mm)
        abi.mpcd_add_momentum(box.h, torch.from_numpy(-dp).to("cuda"))
        box.sync()
        assert np.array_equal(box.state()[1], v1 + (-dp) / mm)


@pytest.mark.parametrize("L,resort_k", [((40, 40, 40), 3), ((33, 29, 31), 0)])
def test_host_state_copy_matches_device_copy(L, resort_k):
    """mpcd_get_state's chunked, overlapped host copy (FP64, 65,536 particles or more; the
    chunk bounds fall at uneven ids here) returns exactly what mpcd_get_state_device gathers,
    after re-sorts scrambled the storage order."""
    torch = pytest.importorskip("torch")
    p = abi.make_params(L, seed=17, resort_k=resort_k)
    with abi.Box(p) as box:
        assert box.n >= 65536
        box.step(7)
        rh, vh = box.state()
        rd = torch.empty((box.n, 3), dtype=torch.float64, device="cuda")
        vd = torch.empty((box.n, 3), dtype=torch.float64, device="cuda")
        abi.mpcd_get_state_device(box.h, rd.data_ptr(), vd.data_ptr())
        box.sync()
        assert np.array_equal(rh, rd.cpu().numpy()) and np.array_equal(vh, vd.cpu().numpy())


@pytest.mark.parametrize("masses", [False, True])
def test_host_state_upload_matches_device_upload(masses):
    """mpcd_set_state's overlapped host upload (FP64, 65,536 particles or more: the positions'
    check and cell-order sort run while the velocities are still being copied) stores exactly
    what mpcd_set_state_device stores: identical storage order, identical steps after it.  A
    state with a bad position or velocity is rejected with the lowest failing id and leaves the
    particles unchanged."""
    torch = pytest.importorskip("torch")
    p = abi.make_params((41, 40, 40), seed=29, resort_k=3)
    rng = np.random.default_rng(30)
    with abi.Box(p) as a, abi.Box(p) as b:
        assert a.n >= 65536
        if masses:
            m = rng.uniform(0.5, 3.0, a.n)
            a.set_masses(m)
            b.set_masses(m)
        r = rng.uniform(0.0, 1.0, (a.n, 3)) * np.array([41.0, 40.0, 40.0])
        v = rng.standard_normal((a.n, 3))
        a.set_state(r, v, 5)
        rd, vd = torch.from_numpy(r).cuda(), torch.from_numpy(v).cuda()
        torch.cuda.synchronize()
        abi.mpcd_set_state_device(b.h, rd.data_ptr(), vd.data_ptr(), 5)
        b.sync()
        del rd, vd
        ra, va = a.state()
        rb, vb = b.state()
        assert np.array_equal(ra, rb) and np.array_equal(va, vb)
        a.step(4)
        b.step(4)
        assert np.array_equal(a.debug_sort()["perm"], b.debug_sort()["perm"])
        sa, sb = a.state(), b.state()
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
        for bad_pos, bad_vel in ((70001, None), (None, 66000), (70001, 66000)):
            rr, vv = r.copy(), v.copy()
            if bad_pos is not None:
                rr[bad_pos, 2] = 40.0                    # on the upper face: outside [0, L a)
            if bad_vel is not None:
                vv[bad_vel, 0] = np.nan
            with pytest.raises(abi.MpcdError) as e:
                a.set_state(rr, vv, 9)
            assert e.value.code == abi.MPCD_ERR_ARG
            assert str(min(x for x in (bad_pos, bad_vel) if x is not None)) in str(e.value)
            now = a.state()
            assert np.array_equal(now[0], sa[0]) and np.array_equal(now[1], sa[1])
        a.step(2)
        b.step(2)
        sa, sb = a.state(), b.state()
        assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
        # two uploads in a row land in alternate buffer sets: both parities against the device path
        for t in (20, 21):
            r2 = rng.uniform(0.0, 1.0, (a.n, 3)) * np.array([41.0, 40.0, 40.0])
            v2 = rng.standard_normal((a.n, 3))
            a.set_state(r2, v2, t)
            rd, vd = torch.from_numpy(r2).cuda(), torch.from_numpy(v2).cuda()
            torch.cuda.synchronize()
            abi.mpcd_set_state_device(b.h, rd.data_ptr(), vd.data_ptr(), t)
            b.sync()
            del rd, vd
            a.step(3)
            b.step(3)
            sa, sb = a.state(), b.state()
            assert np.array_equal(sa[0], sb[0]) and np.array_equal(sa[1], sb[1])
            assert np.array_equal(a.debug_sort()["perm"], b.debug_sort()["perm"])
