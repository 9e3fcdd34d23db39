"""Python access to the FP64 CPU oracle in ``mpcd_oracle.c``.

TEST INFRASTRUCTURE ONLY.  This module and the C code it loads are the slow, plain statement
of one stochastic-rotation-dynamics step (arXiv 2212.11878, Sec. 2 and Sec. 3.1-3.3) that the
CUDA library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference legs may import it; the library never does, and this module imports
nothing from the library.

Arrays follow the C side: positions and velocities are ``(N, 3)`` float64, row-major; ids,
keys, counts, offsets and perm are int32.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liborc.so")
# the same source built with OpenMP: its pragmas run particles and cells in parallel, each
# cell's arithmetic unchanged, so the results are the serial build's bits
OMP_LIB_PATH = os.path.join(BUILD_DIR, "liborc_omp.so")
SOURCES = [os.path.join(HERE, "mpcd_oracle.c")]

TAG_INIT, TAG_SHIFT, TAG_AXIS, TAG_THERMO, TAG_WALL = 0, 1, 2, 3, 4

_lock = threading.Lock()
_lib = None
_omp = False


def build_library(force: bool = False, openmp: bool = False) -> str:
    """Compile ``liborc.so`` with gcc (plain C11, no fast-math, no implicit FMA contraction);
    with ``openmp`` the same source with ``-fopenmp`` as ``liborc_omp.so``."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    path = OMP_LIB_PATH if openmp else LIB_PATH
    newest_src = max(os.path.getmtime(s) for s in SOURCES + [os.path.join(HERE, "mpcd_oracle.h")])
    if not force and os.path.exists(path) and os.path.getmtime(path) >= newest_src:
        return path
    tmp = path + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"] + \
        (["-fopenmp"] if openmp else []) + ["-o", tmp] + SOURCES + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, path)
    return path


def use_openmp(flag: bool) -> None:
    """Route every later call through the OpenMP build (True) or the serial one (False).
    The thread count is OpenMP's (OMP_NUM_THREADS, else all cores)."""
    global _lib, _omp
    with _lock:
        if flag != _omp:
            _lib = None
            _omp = flag


class Params(ctypes.Structure):
    """Mirror of ``orc_params`` (mpcd_oracle.h)."""

    _fields_ = [
        ("L", ctypes.c_int32 * 3),
        ("resort_k", ctypes.c_int32),
        ("a", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("kT", ctypes.c_double),
        ("mass", ctypes.c_double),
        ("ppc", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("seed", ctypes.c_uint64),
        ("walls_z", ctypes.c_int32),
        ("thermostat", ctypes.c_int32),
        ("angular", ctypes.c_int32),
    ]


def make_params(L, a=1.0, dt=0.1, alpha_deg=130.0, kT=1.0, mass=1.0, ppc=10.0, seed=20221211,
                resort_k=0, walls_z=0, g=(0.0, 0.0, 0.0), thermostat=0, alpha=None, angular=0) -> Params:
    p = Params()
    if isinstance(L, int):
        L = (L, L, L)
    p.L[:] = [int(x) for x in L]
    p.resort_k = int(resort_k)
    p.a = float(a)
    p.dt = float(dt)
    p.alpha = float(alpha) if alpha is not None else float(np.deg2rad(alpha_deg))
    p.kT = float(kT)
    p.mass = float(mass)
    p.ppc = float(ppc)
    p.g[:] = [float(x) for x in g]
    p.seed = int(seed)
    p.walls_z = int(walls_z)
    p.thermostat = int(thermostat)
    p.angular = int(angular)
    return p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB lets the mutation tests load a deliberately broken copy
            path = os.environ.get("ORACLE_LIB") or build_library(openmp=_omp)
            L = ctypes.CDLL(path)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            pp = ctypes.POINTER(Params)
            L.orc_philox.argtypes = [u64p, u64p, u64p]
            L.orc_philox.restype = None
            L.orc_u53.argtypes = [ctypes.c_uint64]
            L.orc_u53.restype = ctypes.c_double
            L.orc_num_cells.argtypes = [pp]
            L.orc_num_cells.restype = ctypes.c_int64
            L.orc_shift.argtypes = [pp, ctypes.c_int64, dp]
            L.orc_shift.restype = None
            L.orc_cell_key.argtypes = [pp, dp, dp]
            L.orc_cell_key.restype = ctypes.c_int64
            L.orc_axis.argtypes = [pp, ctypes.c_int64, ctypes.c_int64, dp]
            L.orc_axis.restype = None
            L.orc_mbs_gamma.argtypes = [pp, ctypes.c_int64, ctypes.c_int64, ctypes.c_double]
            L.orc_mbs_gamma.restype = ctypes.c_double
            L.orc_cell_local.argtypes = [pp, dp, dp, dp]
            L.orc_cell_local.restype = None
            L.orc_rotate.argtypes = [dp, ctypes.c_double, dp, dp]
            L.orc_rotate.restype = None
            L.orc_init.argtypes = [pp, ctypes.c_int64, dp, dp]
            L.orc_init.restype = None
            L.orc_step.argtypes = [pp, ctypes.c_int64, ctypes.c_int64, dp, dp, ip, ip, ip, ip, ip, dp, dp]
            L.orc_step.restype = ctypes.c_int
            L.orc_step_m.argtypes = [pp, ctypes.c_int64, ctypes.c_int64, dp, dp, ip, dp, ip, ip, ip, ip, dp, dp]
            L.orc_step_m.restype = ctypes.c_int
            L.orc_presort.argtypes = [pp, ctypes.c_int64, dp, dp, ip, dp]
            L.orc_presort.restype = ctypes.c_int
            _lib = L
        return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if a is not None else None


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox(_u64p(c), _u64p(k), _u64p(out))
    return out


def u53(w: int) -> float:
    return lib().orc_u53(int(w))


def num_cells(p: Params) -> int:
    return int(lib().orc_num_cells(ctypes.byref(p)))


def shift(p: Params, t: int) -> np.ndarray:
    s = np.zeros(3)
    lib().orc_shift(ctypes.byref(p), int(t), _dp(s))
    return s


def cell_key(p: Params, r, s) -> int:
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(3))
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64).reshape(3))
    return int(lib().orc_cell_key(ctypes.byref(p), _dp(r), _dp(s)))


def axis(p: Params, t: int, cell: int) -> np.ndarray:
    n = np.zeros(3)
    lib().orc_axis(ctypes.byref(p), int(t), int(cell), _dp(n))
    return n


def mbs_gamma(p: Params, t: int, cell: int, shape: float) -> float:
    """Gamma(shape, 1) draw of the MBS thermostat for cell `cell` in step t (R22)."""
    return lib().orc_mbs_gamma(ctypes.byref(p), int(t), int(cell), float(shape))


def cell_local(p: Params, r, s) -> np.ndarray:
    """Position of r inside its cell of the grid shifted by s, in cell units (R23)."""
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(3))
    s = np.ascontiguousarray(np.asarray(s, dtype=np.float64).reshape(3))
    out = np.zeros(3)
    lib().orc_cell_local(ctypes.byref(p), _dp(r), _dp(s), _dp(out))
    return out


def rotate(n, alpha: float, u, v) -> np.ndarray:
    n = np.ascontiguousarray(np.asarray(n, dtype=np.float64).reshape(3))
    u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(3))
    out = np.ascontiguousarray(np.array(v, dtype=np.float64).reshape(3))
    lib().orc_rotate(_dp(n), float(alpha), _dp(u), _dp(out))
    return out


def init(p: Params, n: int):
    r = np.zeros((n, 3))
    v = np.zeros((n, 3))
    lib().orc_init(ctypes.byref(p), int(n), _dp(r), _dp(v))
    return r, v


class State:
    """Oracle state: positions, velocities, particle ids and (optionally, R24) per-particle
    masses in storage order, plus the number of completed steps."""

    def __init__(self, r, v, ids=None, t: int = 0, m=None):
        self.r = np.ascontiguousarray(np.array(r, dtype=np.float64).reshape(-1, 3))
        self.v = np.ascontiguousarray(np.array(v, dtype=np.float64).reshape(-1, 3))
        n = self.r.shape[0]
        self.id = (np.arange(n, dtype=np.int32) if ids is None
                   else np.ascontiguousarray(np.asarray(ids, dtype=np.int32)))
        self.m = None if m is None else np.ascontiguousarray(np.array(m, dtype=np.float64).reshape(n))
        self.t = int(t)

    @property
    def n(self) -> int:
        return self.r.shape[0]

    def by_id(self):
        """(r, v) ordered by particle id."""
        order = np.argsort(self.id, kind="stable")
        return self.r[order], self.v[order]

    def masses_by_id(self):
        order = np.argsort(self.id, kind="stable")
        return None if self.m is None else self.m[order]

    def copy(self) -> "State":
        return State(self.r.copy(), self.v.copy(), self.id.copy(), self.t, None if self.m is None else self.m.copy())


def step(p: Params, st: State, debug: bool = False):
    """Advance ``st`` by one step (step index st.t + 1).  With ``debug`` it returns the
    sort and the per-cell moments of that step."""
    n = st.n
    C = num_cells(p)
    out = {}
    keys = counts = offsets = perm = moments = None
    s = np.zeros(3)
    if debug:
        keys = np.zeros(n, np.int32)
        counts = np.zeros(C, np.int32)
        offsets = np.zeros(C + 1, np.int32)
        perm = np.zeros(n, np.int32)
        moments = np.zeros((C, 5))
        out["ids"] = st.id.copy()
    rc = lib().orc_step_m(ctypes.byref(p), n, st.t + 1, _dp(st.r), _dp(st.v), _ip(st.id), _dp(st.m),
                          _ip(keys), _ip(counts), _ip(offsets), _ip(perm), _dp(moments), _dp(s))
    if rc != 0:
        raise RuntimeError("orc_step failed with %d" % rc)
    st.t += 1
    if debug:
        out.update(keys=keys, counts=counts, offsets=offsets, perm=perm, moments=moments)
    out["shift"] = s
    return out


def presort(p: Params, st: State) -> State:
    """Put the storage of ``st`` in cell order of the unshifted grid, stable (reading R25);
    ids and masses move with their particles."""
    rc = lib().orc_presort(ctypes.byref(p), st.n, _dp(st.r), _dp(st.v), _ip(st.id), _dp(st.m))
    if rc != 0:
        raise RuntimeError("orc_presort failed with %d" % rc)
    return st


def run(p: Params, st: State, nsteps: int) -> State:
    for _ in range(nsteps):
        step(p, st)
    return st
