"""The fixed-point cell floor of the FP64 streaming kernels, compiled for the host: wherever
it decides, it equals floor(fl(x - s) / a) (Sec. 2's binning on the shifted grid, the
subtraction rounded once in FP64), including coordinates a few ulps from a face; it leaves
those within 8 / 2^32 cells of a face to the FP64 subtraction and decides every uniform one."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_cell_floor_matches_fp64_definition(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "cell_floor_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_2212_11878_gb300", "csrc"),
                    os.path.join(HERE, "cell_floor_check.cu"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    counts = dict(zip(out.stdout.split()[0::2], map(int, out.stdout.split()[1::2])))
    assert counts["bad"] == 0 and counts["undecided_uniform"] == 0
    assert counts["total"] > 3_000_000 and 0 < counts["undecided"] < counts["total"]
