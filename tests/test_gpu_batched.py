"""GPU checks of the ensemble form (many independent boxes per launch sequence) and of the
autotuner.

An ensemble runs one counting sort over the concatenated cell keys of all boxes; each box
keeps its own parameters and random streams.  Because the per-cell sums are exact
(order-independent), every box of an ensemble must reproduce the same box advanced alone
bit for bit, and no tuning choice may change any result.
"""
import math

import numpy as np
import pytest

from paper_2212_11878_gb300 import abi, inputs

pytestmark = pytest.mark.gpu

BOXES = [
    dict(L=(8, 8, 8), ppc=10, alpha_deg=130, dt=0.1, seed=101),
    dict(L=(12, 12, 12), ppc=5, alpha_deg=60, dt=0.2, seed=102),
    dict(L=(16, 16, 16), ppc=20, alpha_deg=150, dt=0.05, seed=103),
    dict(L=(8, 12, 6), ppc=7, alpha_deg=95, dt=0.1, seed=104),
    dict(L=(4, 4, 4), ppc=13, alpha_deg=110, dt=0.1, seed=105),
]


def box_params(kw):
    return abi.make_params(precision="mixed", **kw)


def test_each_box_equals_the_box_alone():
    params = [box_params(k) for k in BOXES]
    with abi.Box(batch=params) as ens:
        assert abi.mpcd_num_boxes(ens.h) == len(BOXES)
        pb, cb = abi.mpcd_box_offsets(ens.h)
        assert pb[-1] == ens.n and cb[-1] == ens.ncell
        ens.step(6)
        r, v = ens.state()
    for b, p in enumerate(params):
        with abi.Box(p) as one:
            assert one.n == pb[b + 1] - pb[b]
            one.step(6)
            r1, v1 = one.state()
        assert np.array_equal(r[pb[b]:pb[b + 1]], r1), b
        assert np.array_equal(v[pb[b]:pb[b + 1]], v1), b


WALL_BOXES = [
    dict(L=(6, 6, 8), ppc=10, alpha_deg=130, dt=0.1, seed=201, g=(0.01, 0.0, 0.0)),
    dict(L=(8, 4, 10), ppc=15, alpha_deg=100, dt=0.05, seed=202, g=(0.005, 0.002, 0.0)),
    dict(L=(5, 7, 6), ppc=6, alpha_deg=150, dt=0.2, seed=203, g=(0.0, 0.0, 0.0)),
]
SPARSE_BOXES = [  # groups span more than 32 cells here and take the per-cell path
    dict(L=(20, 20, 20), ppc=0.8, alpha_deg=130, dt=0.1, seed=301),
    dict(L=(16, 12, 10), ppc=2, alpha_deg=90, dt=0.2, seed=302),
    dict(L=(6, 6, 6), ppc=12, alpha_deg=120, dt=0.1, seed=303),
]


@pytest.mark.parametrize("boxes,extra", [(WALL_BOXES, dict(walls_z=1, thermostat=1)),
                                         (WALL_BOXES, dict(walls_z=1, thermostat=2)),
                                         (BOXES, dict(thermostat=2)), (SPARSE_BOXES, {}),
                                         (BOXES, dict(angular=1)), (SPARSE_BOXES, dict(angular=1, thermostat=1))],
                         ids=["walls_force_thermostat", "walls_force_mbs", "periodic_mbs", "sparse", "angular",
                              "angular_sparse_thermostat"])
def test_each_box_equals_the_box_alone_other_kinds(boxes, extra):
    params = [abi.make_params(precision="mixed", **k, **extra) for k in boxes]
    with abi.Box(batch=params) as ens:
        pb, _ = abi.mpcd_box_offsets(ens.h)
        ens.step(8)
        r, v = ens.state()
    for b, p in enumerate(params):
        with abi.Box(p) as one:
            one.step(8)
            r1, v1 = one.state()
        assert np.array_equal(r[pb[b]:pb[b + 1]], r1), b
        assert np.array_equal(v[pb[b]:pb[b + 1]], v1), b


def test_ensemble_sort_and_conservation():
    params = [box_params(k) for k in BOXES]
    with abi.Box(batch=params) as ens:
        pb, cb = abi.mpcd_box_offsets(ens.h)
        r0, v0 = ens.state()
        ens.step(1)
        dbg = ens.debug_sort()
        r, v = ens.state()
    keys = np.empty(ens_n := len(dbg["keys"]), np.int64)
    keys[dbg["ids"]] = dbg["keys"]
    assert np.array_equal(dbg["counts"], np.bincount(dbg["keys"], minlength=cb[-1]))
    assert np.array_equal(dbg["perm"], np.argsort(dbg["keys"], kind="stable"))
    for b in range(len(BOXES)):
        sl = slice(pb[b], pb[b + 1])
        assert keys[sl].min() >= cb[b] and keys[sl].max() < cb[b + 1]       # particles stay in their box
        box = np.array(BOXES[b]["L"], float)
        assert np.all(r[sl] >= 0) and np.all(r[sl] < box)
        P0, P1 = v0[sl].sum(axis=0), v[sl].sum(axis=0)
        assert np.abs(P1 - P0).max() < 1e-4 * np.abs(v0[sl]).sum() / 3
        E0, E1 = (v0[sl] ** 2).sum(), (v[sl] ** 2).sum()
        assert abs(E1 / E0 - 1) < 1e-5


def test_recipe_ensemble_runs():
    rec = inputs.batch_recipe(nbox=24, side_choices=(8, 12, 16))
    params = [abi.make_params((s, s, s), ppc=ppc, alpha_deg=al, dt=dt, seed=sd, precision="mixed")
              for s, ppc, al, dt, sd in zip(rec.sides, rec.ppc, rec.alpha_deg, rec.dt, rec.seeds)]
    with abi.Box(batch=params) as ens:
        assert ens.n == rec.n_particles and ens.ncell == rec.cells
        ens.step(20)
        r, v = ens.state()
    assert np.isfinite(v).all()
    assert abs(np.mean(v ** 2) - 1.0) < 0.02


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_autotune_keeps_state_and_results(precision):
    p = abi.make_params((24, 24, 24), precision=precision, seed=7, resort_k=10)
    with abi.Box(p) as a, abi.Box(p) as b:
        a.step(3)
        b.step(3)
        before = a.state()
        best, ms = abi.mpcd_autotune(a.h, trial_steps=2)
        assert ms > 0
        after = a.state()
        assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
        assert abi.mpcd_steps_done(a.h) == 3
        assert abi.mpcd_get_tuning(a.h).as_dict() == best.as_dict()
        a.step(4)
        b.step(4)
        ra, va = a.state()
        rb, vb = b.state()
    assert np.array_equal(ra, rb) and np.array_equal(va, vb)


def test_tunings_give_identical_results():
    p = abi.make_params((20, 20, 20), precision="mixed", seed=9)
    outs = []
    for tg, w in [(96, 2), (224, 4), (160, 2)]:
        with abi.Box(p) as box:
            abi.mpcd_set_tuning(box.h, group_target=tg, warps=w)
            box.step(5)
            outs.append(box.state())
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])
    with abi.Box(p) as box:
        with pytest.raises(abi.MpcdError):
            abi.mpcd_set_tuning(box.h, warps=3)


@pytest.mark.parametrize("extra,boxes", [({}, BOXES), (dict(thermostat=2), BOXES),
                                         (dict(walls_z=1, thermostat=1), WALL_BOXES), ({}, SPARSE_BOXES)],
                         ids=["periodic", "mbs", "walls_thermostat", "sparse"])
def test_one_launch_step_equals_launch_sequence(extra, boxes):
    """The mixed step as one persistent cooperative launch (tuning fuse = 1, the default) and
    as its eight-launch sequence (fuse = 0) give the same bits, over several mpcd_step calls,
    with per-cell moments recorded; the one-launch form launches one kernel per step."""
    params = [abi.make_params(precision="mixed", **k, **extra) for k in boxes]
    outs = []
    for fuse in (1, 0):
        with abi.Box(batch=params) as ens:
            abi.mpcd_set_tuning(ens.h, fuse=fuse)
            abi.mpcd_record_moments(ens.h, True)
            ens.step(1)  # the first step after creation also bins
            l0 = abi.mpcd_launch_count(ens.h)
            for n in (2, 3):
                ens.step(n)
            per_step = (abi.mpcd_launch_count(ens.h) - l0) / 5
            mom, _ = ens.moments()
            outs.append((ens.state(), mom, ens.debug_sort()))
        assert per_step == (1 if fuse else 8)
    (r1, v1), m1, d1 = outs[0]
    (r0, v0), m0, d0 = outs[1]
    assert np.array_equal(r1, r0) and np.array_equal(v1, v0) and np.array_equal(m1, m0)
    for k in ("counts", "offsets"):
        assert np.array_equal(d1[k], d0[k]), k
    # the order inside a cell comes from the scatter's atomics: compare the keys by particle id
    k1 = np.empty(len(d1["keys"]), np.int64)
    k0 = np.empty(len(d0["keys"]), np.int64)
    k1[d1["ids"]] = d1["keys"]
    k0[d0["ids"]] = d0["keys"]
    assert np.array_equal(k1, k0)


def test_one_launch_step_wait_runs_out_with_an_error():
    """Bounded device-side waits: with the test hook set, one block of the one-launch step
    leaves without reaching its grid barriers; the other blocks give up after about a second,
    set the error flag and return, mpcd_sync reports MPCD_ERR_TIMEOUT and poisons the handle,
    and the GPU stays usable (a new box steps normally)."""
    p = abi.make_params((16, 16, 16), precision="mixed", seed=3)
    with abi.Box(p) as box:
        abi.mpcd_set_tuning(box.h, fuse=1)
        box.step(2)
        box.sync()
        assert abi.lib().mpcd_debug_stall_barrier(box.h, 1) == abi.MPCD_OK
        box.step(1)
        with pytest.raises(abi.MpcdError) as e:
            box.sync()
        assert e.value.code == abi.MPCD_ERR_TIMEOUT
        with pytest.raises(abi.MpcdError) as e:
            box.step(1)
        assert e.value.code == abi.MPCD_ERR_STATE
    with abi.Box(p) as fresh, abi.Box(p) as ref:
        abi.mpcd_set_tuning(fresh.h, fuse=1)
        abi.mpcd_set_tuning(ref.h, fuse=0)
        fresh.step(4)
        ref.step(4)
        assert np.array_equal(fresh.state()[1], ref.state()[1])
