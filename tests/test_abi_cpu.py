"""CPU checks of the C-ABI boundary: the library loads, exports every function that
include/mpcd.h declares, the Python mirror of mpcd_params has the C layout, and host-side
argument validation rejects bad parameters before any device work."""
import os
import re
import subprocess

import pytest

from paper_2212_11878_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpcd.h")


@pytest.fixture(scope="module")
def libpath():
    return build.build()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpcd_[a-z0-9_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(abi.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mpcd_[a-z0-9_]+)\b", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    lib = abi.lib()
    for f in declared_functions():
        assert hasattr(lib, f)
    # and no other C-linkage function: internal helpers stay out of the ABI
    c_symbols = set(re.findall(r"\bT ([A-Za-z][A-Za-z0-9_]*)\n", out))
    assert c_symbols <= set(declared_functions()), sorted(c_symbols - set(declared_functions()))


def test_params_layout_matches_c(tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mpcd.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(mpcd_params),'
                    ' offsetof(mpcd_params, a), offsetof(mpcd_params, g), offsetof(mpcd_params, seed),'
                    ' offsetof(mpcd_params, walls_z), offsetof(mpcd_params, angular)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    P = abi.Params
    assert got == [__import__("ctypes").sizeof(P), P.a.offset, P.g.offset, P.seed.offset, P.walls_z.offset,
                   P.angular.offset]


def test_tuning_layout_matches_c(tmp_path):
    prog = tmp_path / "t.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mpcd.h"\n'
                    'int main(void){printf("%zu %zu %zu\\n", sizeof(mpcd_tuning), offsetof(mpcd_tuning, resort_k),'
                    ' offsetof(mpcd_tuning, fuse)); return 0;}\n')
    exe = tmp_path / "t"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    T = abi.Tuning
    assert got == [__import__("ctypes").sizeof(T), T.resort_k.offset, T.fuse.offset]


def test_ensemble_arguments_checked_on_host(libpath):
    a = abi.make_params((4, 4, 4), precision="mixed")
    b = abi.make_params((4, 4, 4), precision="fp64")
    with pytest.raises(abi.MpcdError) as e:
        abi.mpcd_batch_create([a, b])
    assert e.value.code == abi.MPCD_ERR_ARG
    c = abi.make_params((4, 4, 4), precision="mixed", thermostat=1)
    with pytest.raises(abi.MpcdError):
        abi.mpcd_batch_create([a, c])
    bad = abi.make_params((0, 4, 4), precision="mixed")
    with pytest.raises(abi.MpcdError) as e:
        abi.mpcd_batch_create([a, bad])
    assert "box 1" in str(e.value)


def test_version_string(libpath):
    assert "sm_103a" in abi.mpcd_version()


@pytest.mark.parametrize("bad", [
    dict(L=(0, 4, 4)), dict(a=0.0), dict(a=float("nan")), dict(dt=-0.1), dict(kT=0.0), dict(mass=-1.0),
    dict(ppc=-1.0), dict(walls_z=2), dict(walls_z=1, g=(0.0, 0.0, 0.1)), dict(resort_k=-1), dict(precision=7),
    dict(alpha=float("inf")), dict(L=(4096, 4096, 4096)), dict(precision=1, L=(1025, 1025, 1025)),
    dict(thermostat=3), dict(thermostat=-1), dict(angular=2), dict(angular=1, walls_z=1),
])
def test_invalid_params_rejected_on_host(libpath, bad):
    p = abi.make_params(**{**dict(L=(4, 4, 4)), **bad})
    with pytest.raises(abi.MpcdError) as ei:
        abi.mpcd_create(p)
    assert ei.value.code == abi.MPCD_ERR_ARG
    assert abi.mpcd_last_error(None)


def test_null_handle_queries(libpath):
    lib = abi.lib()
    assert lib.mpcd_num_particles(None) == -1
    assert lib.mpcd_step(None, 1) == abi.MPCD_ERR_ARG
    assert lib.mpcd_destroy(None) == 0


def test_handle_less_error_message_is_per_thread(libpath):
    """A failed create (rejected on the host, no device work) leaves its message in the calling
    thread's slot: two threads failing for different reasons each read their own."""
    import ctypes
    import threading

    lib = abi.lib()
    results = {}
    barrier = threading.Barrier(2)

    def worker(name, **bad):
        p = abi.make_params((4, 4, 4), **bad)
        out = ctypes.c_void_p()
        rc = lib.mpcd_create(ctypes.byref(p), ctypes.byref(out))
        barrier.wait()  # both have failed before either reads
        results[name] = (rc, lib.mpcd_last_error(None).decode())

    ts = [threading.Thread(target=worker, args=("kT",), kwargs=dict(kT=-1.0)),
          threading.Thread(target=worker, args=("mass",), kwargs=dict(mass=0.0))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert results["kT"][0] == abi.MPCD_ERR_ARG and "kT" in results["kT"][1]
    assert results["mass"][0] == abi.MPCD_ERR_ARG and "mass" in results["mass"][1]
