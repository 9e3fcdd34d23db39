"""mpcd_step_fp64_noalloc: the FP64 step for callers that may not allocate device memory
(a host framework that owns a fixed device-memory budget, a time-critical loop that must not
take the allocator's locks, a plug-in that is only handed pointers).  Such a caller keeps
its particles in its own device arrays; the library keeps the sort's scratch in one static
device array and allocates nothing.

The test advances the same state twice in a row through the allocation-free entry point
and through the regular handle path (mpcd_create / mpcd_set_state / mpcd_step), and
compares positions and velocities after each call with the parity tolerance (1e-12
relative, tests/parity.py).  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2212_11878_gb300 import abi, inputs
from parity import assert_state_close

pytestmark = pytest.mark.gpu


def _device_soa(torch, a):
    return [torch.from_numpy(np.ascontiguousarray(a[:, d])).to("cuda") for d in range(3)]


def _cell_order(p, r):
    """The storage order mpcd_set_state gives the handle: a stable sort by the cell of each
    position on the unshifted grid (with walls the layer is floor(z / a) + 1).  The caller's
    arrays get the same order, so that both paths sum each cell's members in the same order."""
    c = np.floor(r / p.a).astype(np.int64)
    for d in range(3):
        if d == 2 and p.walls_z:
            c[:, 2] += 1
        else:
            c[:, d] %= p.L[d]
    key = c[:, 0] + p.L[0] * (c[:, 1] + p.L[1] * c[:, 2])
    return np.argsort(key, kind="stable")


@pytest.mark.parametrize("kw", [dict(), dict(thermostat=2), dict(angular=1, thermostat=1),
                                dict(walls_z=1, g=(1e-3, 0.0, 0.0)),
                                dict(walls_z=1, g=(1e-3, 0.0, 0.0), thermostat=1)],
                         ids=["plain", "mbs_thermostat", "angular_thermostat", "walls_force",
                              "walls_force_thermostat"])
def test_noalloc_step_matches_handle_path(kw):
    """With a thermostat or walls both paths take the per-cell kernel; plain boxes compare
    the per-cell kernel with the dense pair."""
    torch = pytest.importorskip("torch")
    L = (12, 10, 8)
    p = abi.make_params(L, resort_k=0, seed=4242, **kw)
    n = int(round(p.ppc * 12 * 10 * 8))
    r, v = inputs.uniform_gaussian_state(L, n, 99)
    t0 = 5
    order = _cell_order(p, r)
    x = _device_soa(torch, r[order])
    u = _device_soa(torch, v[order])
    stream = torch.cuda.current_stream().cuda_stream
    with abi.Box(p) as box:
        box.set_state(r, v, t0)
        for call in range(2):
            abi.mpcd_step_fp64_noalloc(p, t0 + call, n, *x, *u, stream=stream)
            torch.cuda.synchronize()
            box.step(1)
            r_ref, v_ref = box.state()
            r_na = np.empty_like(r)
            v_na = np.empty_like(v)
            r_na[order] = np.stack([a.cpu().numpy() for a in x], axis=1)
            v_na[order] = np.stack([a.cpu().numpy() for a in u], axis=1)
            assert_state_close(r_na, v_na, r_ref, v_ref, p, what="no-alloc call %d" % (call + 1))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    p = abi.make_params((8, 8, 8))
    with pytest.raises(abi.MpcdError) as e:
        abi.mpcd_step_fp64_noalloc(p, 0, abi.MPCD_NOALLOC_MAX_PARTICLES + 1, 1, 1, 1, 1, 1, 1)
    assert e.value.code == abi.MPCD_ERR_ARG and "MPCD_NOALLOC_MAX_PARTICLES" in str(e.value)
    big = abi.make_params((64, 64, 64), ppc=1.0)
    with pytest.raises(abi.MpcdError) as e:
        abi.mpcd_step_fp64_noalloc(big, 0, 1000, 1, 1, 1, 1, 1, 1)
    assert e.value.code == abi.MPCD_ERR_ARG and "MPCD_NOALLOC_MAX_CELLS" in str(e.value)
    # walls add a cell layer: 64 x 64 x 32 fits the scratch exactly, with walls it does not
    edge = abi.make_params((64, 64, 32), ppc=0.0)
    abi.mpcd_step_fp64_noalloc(edge, 0, 0, 0, 0, 0, 0, 0, 0)
    walled = abi.make_params((64, 64, 32), ppc=0.0, walls_z=1)
    with pytest.raises(abi.MpcdError) as e:
        abi.mpcd_step_fp64_noalloc(walled, 0, 0, 0, 0, 0, 0, 0, 0)
    assert e.value.code == abi.MPCD_ERR_ARG and "MPCD_NOALLOC_MAX_CELLS" in str(e.value)
