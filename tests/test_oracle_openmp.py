"""The OpenMP build of the oracle (the same C source, its pragmas run particles and cells in
parallel) must give the serial build's bits: every cell's arithmetic is unchanged, so the
all-cores CPU baseline times the same computation as the single-core one."""
import numpy as np
import pytest

from paper_2212_11878_gb300 import inputs

CASES = {
    "periodic_resort": dict(L=(9, 8, 7), resort_k=2),
    "walls_mbs": dict(L=(6, 5, 8), walls_z=1, g=(0.01, 0.0, 0.0), thermostat=2, ppc=12),
    "angular_thermostat": dict(L=(7, 6, 5), angular=1, thermostat=1),
}


def _run(orc, kw, steps, masses):
    p = orc.make_params(seed=55, **kw)
    L = tuple(kw["L"])
    n = int(round(p.ppc * np.prod(L)))
    r, v = inputs.uniform_gaussian_state(L, n, 9)
    m = np.random.default_rng(2).uniform(0.5, 3.0, n) if masses else None
    st = orc.presort(p, orc.State(r, v, m=m))
    outs = [orc.step(p, st, debug=True) for _ in range(steps)]
    return st, outs


@pytest.mark.parametrize("name", list(CASES))
def test_openmp_build_is_bit_identical(orc, name, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "4")
    orc.build_library(openmp=True)
    kw = CASES[name]
    try:
        orc.use_openmp(False)
        a, oa = _run(orc, kw, 4, masses=name != "walls_mbs")
        orc.use_openmp(True)
        b, ob = _run(orc, kw, 4, masses=name != "walls_mbs")
    finally:
        orc.use_openmp(False)
    assert np.array_equal(a.r, b.r) and np.array_equal(a.v, b.v) and np.array_equal(a.id, b.id)
    for x, y in zip(oa, ob):
        for k in ("keys", "counts", "offsets", "perm", "moments", "shift"):
            assert np.array_equal(x[k], y[k]), k
