"""CPU check (no GPU) of BlockWalk, the division-free index walk of the
subset kernel's update pass and gather (csrc/haf_internal.h):
tests/native/block_walk.cu compares it with (e / L, e % L) for every column
count, group width and lane the kernel can use.  Built with nvcc for the
host; it launches nothing."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_block_walk_matches_division(tmp_path):
    nvcc = next((c for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc") if c and os.path.exists(c)), None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "block_walk")
    build = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                            "-I", os.path.join(ROOT, "include"),
                            os.path.join(ROOT, "tests", "native", "block_walk.cu"), "-o", exe],
                           capture_output=True, text=True, timeout=600)
    assert build.returncode == 0, build.stderr[-2000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and "block walk ok" in run.stdout, run.stdout[-2000:]
