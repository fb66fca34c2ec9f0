"""CPU checks (no GPU) of two host-and-device helpers of
csrc/haf_internal.h, built with nvcc for the host (they launch nothing):
  - BlockWalk, the division-free index walk of the subset kernel's update
    pass and gather (tests/native/block_walk.cu): equal to (e / L, e % L)
    for every column count, group width and lane the kernel can use;
  - subset_layout, the per-subset shared-memory map
    (tests/native/subset_layout_check.cu): regions in order, aligned, and
    within the total, the loop hafnian's reuse of W and P only where they
    hold h + 1 elements."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build_and_run(tmp_path, name):
    nvcc = next((c for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc") if c and os.path.exists(c)), None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / name)
    build = subprocess.run([nvcc, "-std=c++17", "-O2", "-gencode", "arch=compute_103a,code=sm_103a",
                            "-I", os.path.join(ROOT, "include"),
                            os.path.join(ROOT, "tests", "native", name + ".cu"), "-o", exe],
                           capture_output=True, text=True, timeout=600)
    assert build.returncode == 0, build.stderr[-2000:]
    return subprocess.run([exe], capture_output=True, text=True, timeout=300)


def test_block_walk_matches_division(tmp_path):
    run = _build_and_run(tmp_path, "block_walk")
    assert run.returncode == 0 and "block walk ok" in run.stdout, run.stdout[-2000:]


def test_subset_layout_invariants(tmp_path):
    run = _build_and_run(tmp_path, "subset_layout_check")
    assert run.returncode == 0 and "layout ok" in run.stdout, run.stdout[-2000:]
