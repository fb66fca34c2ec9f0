"""The product path has no CPU fallback: without a usable CUDA library or
GPU every compute call raises, and the package never reaches the oracle.

These run on the CPU only.  A GPU-less process is the natural test bed:
any call that returned a number here would have to come from host code."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1805_12498_gb300")


def _gpu_present() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def test_package_sources_never_name_the_oracle():
    """No module of the library imports, loads or runs anything under oracle/."""
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|.*liboracle)", re.M)
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".c", ".cpp")):
                with open(os.path.join(dirpath, f)) as fh:
                    assert not pat.search(fh.read()), os.path.join(dirpath, f)


_PROBE = r"""
import sys, numpy as np
import paper_1805_12498_gb300 as hg
A = np.ones((8, 8))
calls = {
    "haf": lambda: hg.haf(A),
    "lhaf": lambda: hg.lhaf(A),
    "haf_info real": lambda: hg.haf_info(A, real=True),
    "fp32": lambda: hg.haf(A, precision="fp32"),
    "batched": lambda: hg.haf_batched([A, A[:4, :4]]),
    "terms": lambda: hg.haf_terms(A, np.array([1, 3], dtype=np.uint64)),
    "lowrank": lambda: hg.haf_lowrank(np.ones((8, 1))),
    "part": lambda: hg.haf_part(A, 0, 2),
}
for name, f in calls.items():
    try:
        v = f()
    except hg.HafError as e:
        print(name, "raised", e.code)
    else:
        print(name, "RETURNED", v)
print("oracle loaded:", "oracle" in sys.modules)
"""


@pytest.mark.skipif(_gpu_present(), reason="needs a process without a GPU")
def test_every_compute_call_raises_without_a_gpu():
    r = subprocess.run([sys.executable, "-c", _PROBE], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = r.stdout.strip().splitlines()
    assert lines[-1] == "oracle loaded: False"
    results = lines[:-1]
    assert len(results) == 8
    for line in results:
        assert "RETURNED" not in line, line
        assert line.endswith("raised -3"), line  # HAF_ECUDA


_MISSING = r"""
import sys, numpy as np
from paper_1805_12498_gb300 import _native, build
def no_toolkit(*a, **k):
    raise RuntimeError("nvcc not found")
build.build = no_toolkit
build.LIB = sys.argv[1]
import paper_1805_12498_gb300 as hg
try:
    hg.haf(np.ones((4, 4)))
except RuntimeError as e:
    print("raised:", e)
else:
    print("RETURNED")
try:
    _native.lib(build_if_missing=False)
except RuntimeError as e:
    print("raised:", e)
else:
    print("LOADED")
print("oracle loaded:", "oracle" in sys.modules)
"""


def test_missing_library_raises(tmp_path):
    """With the library absent and no toolkit to build it, calls raise."""
    missing = str(tmp_path / "libhafnian_gb300.so")
    r = subprocess.run([sys.executable, "-c", _MISSING, missing], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    out = r.stdout.strip().splitlines()
    assert out[0] == "raised: nvcc not found"
    assert out[1].startswith("raised: CUDA library") and "missing" in out[1]
    assert out[2] == "oracle loaded: False"


def test_binding_only_marshals():
    """The Python front end holds no hafnian arithmetic: none of the
    method's steps (Householder, La Budde, the det^{-1/2} series, the
    matching sum) appears in it, and it calls no numpy linear algebra."""
    for f in ("__init__.py", "_native.py"):
        with open(os.path.join(PKG, f)) as fh:
            src = fh.read()
        for banned in ("np.linalg", "scipy", "eigvals", "householder", "labudde", "np.poly"):
            assert banned not in src, (f, banned)
