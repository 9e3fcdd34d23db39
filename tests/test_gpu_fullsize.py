"""Parity at the sizes the bench runs, in the launch configuration it times (CUDA-graph
replay of mpcd_step).

* FP64, 128^3 cells, 20,971,520 particles, re-sort every 10 steps: two steps from the same
  state through the library and the oracle, the first a re-sort step.  At this size every
  grid-stride loop of the FP64 kernels runs several sweeps (the grids are capped at 152 x 64
  blocks), which the small parity cases never reach.  Keys, counts, offsets, perm and ids
  bit-exact; positions and velocities within 1e-12 relative.
* The mixed-form ensemble of 32 uneven boxes: one step from a state every box represents
  exactly, each box against the oracle run on that box alone, at the mixed form's one-step
  bounds.
"""
import numpy as np
import pytest

from paper_2212_11878_gb300 import abi, inputs
from parity import assert_mixed_one_step, assert_sort_equal, assert_state_close, oracle_params

pytestmark = pytest.mark.gpu


def test_fp64_128cubed_resort_and_plain_step_match_oracle(orc):
    w = inputs.WORKLOADS["fp64_L128"]
    p = abi.params_from_workload(w)
    assert p.resort_k == 10 and w.n_particles == 20971520
    r, v = inputs.uniform_gaussian_state(tuple(w.L), w.n_particles, 808)
    t0 = 9  # step 10 re-sorts the storage, step 11 does not
    op = oracle_params(orc, p)
    orc.use_openmp(True)  # the OpenMP build: the serial build's bits (tests/test_oracle_openmp.py)
    try:
        st = orc.presort(op, orc.State(r, v, t=t0))
        with abi.Box(p) as box:
            box.set_state(r, v, t0)
            for k in range(2):
                box.step(1)
                ref = orc.step(op, st, debug=True)
                assert_sort_equal(box.debug_sort(), ref)
                rg, vg = box.state()
                rr, vr = st.by_id()
                assert_state_close(rg, vg, rr, vr, p, what="128^3 step %d" % (t0 + k + 1))
    finally:
        orc.use_openmp(False)


def quantize(r, v, L, a=1.0):
    """A state the mixed form stores exactly: r = (c + f) a with f an FP32 in [0, 1)."""
    q = r / a
    c = np.floor(q)
    f = (q - c).astype(np.float32).astype(np.float64)
    up = f >= 1.0
    f[up] = 0.0
    c[up] += 1
    c = np.mod(c, np.asarray(L))
    return (c + f) * a, v.astype(np.float32).astype(np.float64)


def test_ensemble_boxes_match_oracle_one_step(orc):
    rec = inputs.batch_workload("batched_32")
    params = abi.params_from_recipe(rec)
    states = []
    for b, p in enumerate(params):
        L = tuple(p.L)
        n = int(round(p.ppc * np.prod(L)))
        states.append(quantize(*inputs.uniform_gaussian_state(L, n, 500 + b), L, p.a))
    r0 = np.concatenate([s[0] for s in states])
    v0 = np.concatenate([s[1] for s in states])
    t0 = 4
    with abi.Box(batch=params) as ens:
        pb, cb = abi.mpcd_box_offsets(ens.h)
        assert ens.n == len(r0)
        ens.set_state(r0, v0, t0)
        ens.step(1)
        dbg = ens.debug_sort()
        rg, vg = ens.state()
    keys = np.empty(len(r0), np.int64)
    keys[dbg["ids"]] = dbg["keys"]
    for b, p in enumerate(params):
        sl = slice(pb[b], pb[b + 1])
        st = orc.State(*states[b], t=t0)
        ref = orc.step(oracle_params(orc, p), st, debug=True)
        rr, vr = st.by_id()
        ko = np.empty(st.n, np.int64)
        ko[ref["ids"]] = ref["keys"]
        assert_mixed_one_step(p, keys[sl] - cb[b], ko, rg[sl], vg[sl], rr, vr, ref["shift"], cb[b + 1] - cb[b],
                              what="box %d (side %d, ppc %g)" % (b, p.L[0], p.ppc))
