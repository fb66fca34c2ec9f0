"""CPU check (no GPU) of the low-rank step kernels' index logic:
tests/native/lowrank_walks.cu includes csrc/haf_lowrank.cu, whose rank and
walk helpers are __host__ __device__, and runs them on the host against
brute-force enumeration of compositions (bars of every rank on every
lane's walk, predecessor ranks, cube offsets and steps).  Built with nvcc
for the host; it launches nothing."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_lowrank_walks_against_enumeration(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "lowrank_walks")
    src = os.path.join(ROOT, "tests", "native", "lowrank_walks.cu")
    build = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                            "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                           capture_output=True, text=True, timeout=900)
    assert build.returncode == 0, build.stderr[-2000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert run.returncode == 0 and "walks ok" in run.stdout, run.stdout[-2000:]
