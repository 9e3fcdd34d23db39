"""ctypes binding of libmpcd (include/mpcd.h).  Argument marshalling only: every step of the
SRD computation runs in the library's CUDA kernels.

Functions carry the C names (``mpcd_create``, ``mpcd_step``, ...).  Host arrays are numpy
float64 arrays of shape (N, 3); device arrays are passed as integer pointers (for example
``tensor.data_ptr()`` of a CUDA tensor).  Every non-zero return code raises
:class:`MpcdError` with the library's message.  If ``lib/libmpcd.so`` has not been built,
:func:`lib` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libmpcd.so")

MPCD_OK, MPCD_ERR_ARG, MPCD_ERR_CUDA, MPCD_ERR_OOM, MPCD_ERR_TIMEOUT, MPCD_ERR_STATE = 0, -1, -2, -3, -4, -5
MPCD_FP64, MPCD_MIXED = 0, 1

# every symbol include/mpcd.h declares
EXPORTS = [
    "mpcd_create", "mpcd_batch_create", "mpcd_destroy", "mpcd_set_stream", "mpcd_step", "mpcd_sync",
    "mpcd_num_particles", "mpcd_num_cells", "mpcd_steps_done", "mpcd_num_boxes", "mpcd_get_state",
    "mpcd_set_state", "mpcd_get_state_device", "mpcd_set_state_device", "mpcd_record_moments",
    "mpcd_cell_moments", "mpcd_debug_sort", "mpcd_timing", "mpcd_timing_read", "mpcd_launch_count",
    "mpcd_last_error", "mpcd_version", "mpcd_step_fp64_noalloc", "mpcd_box_offsets", "mpcd_get_tuning",
    "mpcd_set_tuning", "mpcd_autotune", "mpcd_set_masses", "mpcd_get_masses", "mpcd_measure_fp64_rate",
    "mpcd_add_momentum", "mpcd_add_momentum_device", "mpcd_debug_stall_barrier",
]
MPCD_NOALLOC_MAX_PARTICLES = 1 << 19
MPCD_NOALLOC_MAX_CELLS = 1 << 17


class MpcdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("libmpcd error %d: %s" % (code, msg))
        self.code = code


class Params(ctypes.Structure):
    """Mirror of ``mpcd_params``."""

    _fields_ = [
        ("L", ctypes.c_int32 * 3),
        ("precision", ctypes.c_int32),
        ("a", ctypes.c_double),
        ("ppc", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("seed", ctypes.c_uint64),
        ("walls_z", ctypes.c_int32),
        ("thermostat", ctypes.c_int32),
        ("resort_k", ctypes.c_int32),
        ("angular", ctypes.c_int32),
    ]


class Tuning(ctypes.Structure):
    """Mirror of ``mpcd_tuning``."""

    _fields_ = [("group_target", ctypes.c_int32), ("warps", ctypes.c_int32), ("resort_k", ctypes.c_int32),
                ("fuse", ctypes.c_int32)]

    def as_dict(self):
        return {"group_target": self.group_target, "warps": self.warps, "resort_k": self.resort_k, "fuse": self.fuse}


def make_params(L, a=1.0, ppc=10.0, dt=0.1, alpha_deg=130.0, kT=1.0, mass=1.0, seed=20221211,
                precision="fp64", walls_z=0, g=(0.0, 0.0, 0.0), thermostat=0, resort_k=1, alpha=None,
                angular=0) -> Params:
    p = Params()
    if isinstance(L, int):
        L = (L, L, L)
    p.L[:] = [int(x) for x in L]
    p.precision = {"fp64": MPCD_FP64, "mixed": MPCD_MIXED}[precision] if isinstance(precision, str) else int(precision)
    p.a = float(a)
    p.ppc = float(ppc)
    p.dt = float(dt)
    p.alpha = float(alpha) if alpha is not None else math.radians(alpha_deg)
    p.kT = float(kT)
    p.mass = float(mass)
    p.g[:] = [float(x) for x in g]
    p.seed = int(seed)
    p.walls_z = int(walls_z)
    p.thermostat = int(thermostat)
    p.resort_k = int(resort_k)
    p.angular = int(angular)
    return p


def params_from_workload(w, **override) -> Params:
    kw = dict(L=w.L, a=w.a, ppc=w.ppc, dt=w.dt, alpha_deg=w.alpha_deg, kT=w.kT, mass=w.mass, seed=w.seed,
              precision=w.precision, walls_z=w.walls_z, g=w.g, thermostat=w.thermostat, resort_k=w.resort_k,
              angular=getattr(w, "angular", 0))
    kw.update(override)
    return make_params(**kw)


def params_from_recipe(rec, precision="mixed", kT=1.0, mass=1.0):
    """One Params per box of an ensemble recipe (paper_2212_11878_gb300.inputs.BatchRecipe)."""
    return [make_params((s, s, s), ppc=ppc, alpha_deg=al, dt=dt, seed=sd, precision=precision, kT=kT, mass=mass)
            for s, ppc, al, dt, sd in zip(rec.sides, rec.ppc, rec.alpha_deg, rec.dt, rec.seeds)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libmpcd.so (built by paper_2212_11878_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libmpcd.so is not built (%s); run python -m paper_2212_11878_gb300.build" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            H = ctypes.c_void_p
            i32, i64, dp, ip = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
            sig = {
                "mpcd_create": ([ctypes.POINTER(Params), ctypes.POINTER(H)], ctypes.c_int),
                "mpcd_batch_create": ([i32, ctypes.POINTER(Params), ctypes.POINTER(H)], ctypes.c_int),
                "mpcd_destroy": ([H], ctypes.c_int),
                "mpcd_set_stream": ([H, ctypes.c_void_p], ctypes.c_int),
                "mpcd_step": ([H, i64], ctypes.c_int),
                "mpcd_sync": ([H], ctypes.c_int),
                "mpcd_num_particles": ([H], i64),
                "mpcd_num_cells": ([H], i64),
                "mpcd_steps_done": ([H], i64),
                "mpcd_num_boxes": ([H], i32),
                "mpcd_get_state": ([H, dp, dp], ctypes.c_int),
                "mpcd_set_state": ([H, i64, dp, dp, i64], ctypes.c_int),
                "mpcd_set_masses": ([H, i64, dp], ctypes.c_int),
                "mpcd_get_masses": ([H, dp], ctypes.c_int),
                "mpcd_get_state_device": ([H, dp, dp], ctypes.c_int),
                "mpcd_set_state_device": ([H, i64, dp, dp, i64], ctypes.c_int),
                "mpcd_record_moments": ([H, i32], ctypes.c_int),
                "mpcd_cell_moments": ([H, dp, dp], ctypes.c_int),
                "mpcd_debug_sort": ([H, ip, ip, ip, ip, ip], ctypes.c_int),
                "mpcd_timing": ([H, i32], ctypes.c_int),
                "mpcd_timing_read": ([H, i32, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
                "mpcd_launch_count": ([H], i64),
                "mpcd_last_error": ([H], ctypes.c_char_p),
                "mpcd_version": ([], ctypes.c_char_p),
                "mpcd_measure_fp64_rate": ([dp], ctypes.c_int),
                "mpcd_add_momentum": ([H, i64, dp], ctypes.c_int),
                "mpcd_debug_stall_barrier": ([H, i32], ctypes.c_int),
                "mpcd_add_momentum_device": ([H, i64, dp], ctypes.c_int),
                "mpcd_step_fp64_noalloc": ([ctypes.POINTER(Params), i64, i64] + [dp] * 6 + [ctypes.c_void_p],
                                           ctypes.c_int),
                "mpcd_box_offsets": ([H, dp, dp], ctypes.c_int),
                "mpcd_get_tuning": ([H, ctypes.POINTER(Tuning)], ctypes.c_int),
                "mpcd_set_tuning": ([H, ctypes.POINTER(Tuning)], ctypes.c_int),
                "mpcd_autotune": ([H, i32, ctypes.POINTER(Tuning), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
        return _lib


def _check(rc: int, h=None) -> int:
    if rc < 0:
        msg = lib().mpcd_last_error(h)
        raise MpcdError(rc, msg.decode() if msg else "")
    return rc


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _host_f64(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(n, 3))
    return a


# ---- the C entry points, one Python function each ----
def mpcd_create(params: Params):
    h = ctypes.c_void_p()
    _check(lib().mpcd_create(ctypes.byref(params), ctypes.byref(h)))
    return h


def mpcd_batch_create(params_list):
    arr = (Params * len(params_list))(*params_list)
    h = ctypes.c_void_p()
    _check(lib().mpcd_batch_create(len(params_list), arr, ctypes.byref(h)))
    return h


def mpcd_destroy(h):
    return _check(lib().mpcd_destroy(h))


def mpcd_set_stream(h, stream_handle: int):
    return _check(lib().mpcd_set_stream(h, stream_handle), h)


def mpcd_step(h, nsteps: int):
    return _check(lib().mpcd_step(h, int(nsteps)), h)


def mpcd_sync(h):
    return _check(lib().mpcd_sync(h), h)


def mpcd_num_particles(h) -> int:
    return int(lib().mpcd_num_particles(h))


def mpcd_num_cells(h) -> int:
    return int(lib().mpcd_num_cells(h))


def mpcd_steps_done(h) -> int:
    return int(lib().mpcd_steps_done(h))


def mpcd_num_boxes(h) -> int:
    return int(lib().mpcd_num_boxes(h))


def mpcd_get_state(h, r=None, v=None):
    n = mpcd_num_particles(h)
    r = np.empty((n, 3)) if r is None else r
    v = np.empty((n, 3)) if v is None else v
    _check(lib().mpcd_get_state(h, _ptr(r), _ptr(v)), h)
    return r, v


def mpcd_set_masses(h, m):
    """Per-particle masses in particle-id order (FP64 form); None restores the box mass."""
    n = mpcd_num_particles(h)
    if m is None:
        _check(lib().mpcd_set_masses(h, n, None), h)
        return
    m = np.ascontiguousarray(np.asarray(m, dtype=np.float64).reshape(n))
    _check(lib().mpcd_set_masses(h, n, _ptr(m)), h)


def mpcd_get_masses(h):
    m = np.empty(mpcd_num_particles(h))
    _check(lib().mpcd_get_masses(h, _ptr(m)), h)
    return m


def mpcd_set_state(h, r, v, t: int = 0):
    n = mpcd_num_particles(h)
    if not (hasattr(r, "data_ptr") and hasattr(v, "data_ptr")):
        r, v = _host_f64(r, n), _host_f64(v, n)
    return _check(lib().mpcd_set_state(h, n, _ptr(r), _ptr(v), int(t)), h)


def mpcd_get_state_device(h, r_dev, v_dev):
    return _check(lib().mpcd_get_state_device(h, _ptr(r_dev), _ptr(v_dev)), h)


def mpcd_set_state_device(h, r_dev, v_dev, t: int = 0):
    return _check(lib().mpcd_set_state_device(h, mpcd_num_particles(h), _ptr(r_dev), _ptr(v_dev), int(t)), h)


def mpcd_record_moments(h, enable: bool = True):
    return _check(lib().mpcd_record_moments(h, 1 if enable else 0), h)


def mpcd_cell_moments(h):
    C = mpcd_num_cells(h)
    out = np.empty((C, 5))
    s = np.empty(3)
    _check(lib().mpcd_cell_moments(h, _ptr(out), _ptr(s)), h)
    return out, s


def mpcd_debug_sort(h):
    n, C = mpcd_num_particles(h), mpcd_num_cells(h)
    keys = np.empty(n, np.int32)
    counts = np.empty(C, np.int32)
    offsets = np.empty(C + 1, np.int32)
    perm = np.empty(n, np.int32)
    ids = np.empty(n, np.int32)
    _check(lib().mpcd_debug_sort(h, _ptr(keys), _ptr(counts), _ptr(offsets), _ptr(perm), _ptr(ids)), h)
    return dict(keys=keys, counts=counts, offsets=offsets, perm=perm, ids=ids)


def mpcd_timing(h, enable: bool = True):
    return _check(lib().mpcd_timing(h, 1 if enable else 0), h)


def mpcd_timing_read(h, nmax: int = 32):
    names = (ctypes.c_char_p * nmax)()
    ms = (ctypes.c_double * nmax)()
    launches = (ctypes.c_int64 * nmax)()
    k = _check(lib().mpcd_timing_read(h, nmax, names, ms, launches), h)
    return {names[i].decode(): (ms[i], int(launches[i])) for i in range(k)}


def mpcd_launch_count(h) -> int:
    return int(lib().mpcd_launch_count(h))


def mpcd_last_error(h=None) -> str:
    m = lib().mpcd_last_error(h)
    return m.decode() if m else ""


def mpcd_version() -> str:
    return lib().mpcd_version().decode()


def mpcd_add_momentum(h, dp):
    """v_i += dp_i / m_i for every particle (dp: (N, 3) FP64 in particle-id order, host or device)."""
    n = mpcd_num_particles(h)
    if hasattr(dp, "data_ptr"):
        assert tuple(dp.shape) == (n, 3) and dp.is_contiguous()
        return _check(lib().mpcd_add_momentum_device(h, n, dp.data_ptr()), h)
    a = np.ascontiguousarray(dp, dtype=np.float64)
    if a.shape != (n, 3):
        raise ValueError("dp must have shape (N, 3)")
    return _check(lib().mpcd_add_momentum(h, n, a.ctypes.data), h)


def mpcd_measure_fp64_rate() -> float:
    """FP64 FMAs per second (counted per lane) of the current GPU, measured."""
    out = ctypes.c_double(0.0)
    rc = lib().mpcd_measure_fp64_rate(ctypes.byref(out))
    if rc != MPCD_OK:
        raise MpcdError(rc, "FP64 rate probe failed")
    return out.value


def mpcd_step_fp64_noalloc(params: Params, t: int, n: int, x, y, z, vx, vy, vz, stream=None):
    """One FP64 step on caller-owned device arrays; the library allocates nothing."""
    return _check(lib().mpcd_step_fp64_noalloc(ctypes.byref(params), int(t), int(n), _ptr(x), _ptr(y), _ptr(z),
                                               _ptr(vx), _ptr(vy), _ptr(vz), stream))


def mpcd_box_offsets(h):
    nb = mpcd_num_boxes(h)
    pb = np.empty(nb + 1, np.int64)
    cb = np.empty(nb + 1, np.int64)
    _check(lib().mpcd_box_offsets(h, _ptr(pb), _ptr(cb)), h)
    return pb, cb


def mpcd_get_tuning(h) -> Tuning:
    t = Tuning()
    _check(lib().mpcd_get_tuning(h, ctypes.byref(t)), h)
    return t


def mpcd_set_tuning(h, group_target=None, warps=None, resort_k=None, fuse=None):
    t = mpcd_get_tuning(h)
    if fuse is not None:
        t.fuse = int(fuse)
    if group_target is not None:
        t.group_target = int(group_target)
    if warps is not None:
        t.warps = int(warps)
    if resort_k is not None:
        t.resort_k = int(resort_k)
    return _check(lib().mpcd_set_tuning(h, ctypes.byref(t)), h)


def mpcd_autotune(h, trial_steps: int = 5):
    """Returns (best Tuning, best ms per step); the state is left unchanged."""
    t = Tuning()
    ms = ctypes.c_double()
    _check(lib().mpcd_autotune(h, int(trial_steps), ctypes.byref(t), ctypes.byref(ms)), h)
    return t, ms.value


class Box:
    """Owns one handle; convenience methods over the functions above."""

    def __init__(self, params: Params = None, batch=None):
        self.h = mpcd_batch_create(batch) if batch is not None else mpcd_create(params)

    def close(self):
        if self.h:
            mpcd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return mpcd_num_particles(self.h)

    @property
    def ncell(self) -> int:
        return mpcd_num_cells(self.h)

    def step(self, nsteps: int = 1):
        mpcd_step(self.h, nsteps)

    def sync(self):
        mpcd_sync(self.h)

    def state(self):
        return mpcd_get_state(self.h)

    def set_state(self, r, v, t: int = 0):
        mpcd_set_state(self.h, r, v, t)

    def set_masses(self, m):
        mpcd_set_masses(self.h, m)

    def moments(self):
        return mpcd_cell_moments(self.h)

    def debug_sort(self):
        return mpcd_debug_sort(self.h)
