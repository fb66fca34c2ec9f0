"""The C-ABI library builds, loads and exports every function that
include/*.h declares.  No compute calls (this runs without a GPU)."""
import ctypes
import math
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*[\s\*]+([a-z_][a-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared_functions()
    for must in ("haf_c128", "lhaf_c128", "haf_f64", "lhaf_f64", "haf_c128_batched",
                 "lhaf_c128_batched", "haf_launch", "haf_workspace_bytes", "haf_terms_c128",
                 "haf_eval", "haf_batched", "haf_terms", "haf_tune", "haf_tune_set", "haf_batched_tune",
                 "haf_server_create", "haf_server_submit", "haf_server_poll", "haf_server_destroy",
                 "haf_part", "haf_combine", "haf_launch_noalloc", "haf_lowrank_c128",
                 "haf_lowrank_workspace_bytes", "haf_lowrank_launch"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1805_12498_gb300 import _native
    L = _native.lib()  # builds in-tree with nvcc if needed (no GPU required)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, f"not exported: {missing}"


def test_library_is_in_tree_and_sm103a():
    from paper_1805_12498_gb300 import _native, build
    path = _native.lib_path()
    assert os.path.dirname(path).startswith(ROOT)
    assert any("compute_103a" in a for a in build.ARCH)


def test_bad_arguments_fail_without_gpu_work():
    """Argument checks run before any CUDA call."""
    from paper_1805_12498_gb300 import _native
    L = _native.lib()
    out = (ctypes.c_double * 2)()
    assert L.haf_c128(None, 4, out, None) == _native.HAF_EINVAL
    assert L.haf_c128(None, -1, out, None) == _native.HAF_EINVAL
    assert L.haf_c128(None, 1000, out, None) == _native.HAF_EINVAL
    assert L.haf_launch(None, 5, 0, None, None, 0, None) == _native.HAF_EINVAL
    assert b"n must be even" in L.haf_last_error()
    A = (ctypes.c_double * 32)()
    assert L.haf_eval(A, 4, 1 << 7, out, None) == _native.HAF_EINVAL
    assert b"unknown flags" in L.haf_last_error()
    assert L.haf_tune_set(16, 0, 5, 8) == _native.HAF_EINVAL
    assert L.haf_tune_set(16, 0, 8, 0) == _native.HAF_EINVAL
    assert L.haf_tune_set(15, 0, 8, 8) == _native.HAF_EINVAL
    r = _native.TuneResult()
    assert L.haf_tune(16, 0, 0, ctypes.byref(r)) == _native.HAF_EINVAL
    assert L.haf_lowrank_c128(None, 4, 2, out, None) == _native.HAF_EINVAL
    assert L.haf_lowrank_c128(A, 4, 0, out, None) == _native.HAF_EINVAL
    assert L.haf_lowrank_c128(A, 4, 17, out, None) == _native.HAF_EINVAL
    # device-pointer form: argument checks come before any CUDA call (the
    # pointer values below are never dereferenced)
    assert L.haf_lowrank_workspace_bytes(5, 2) == 0 and L.haf_lowrank_workspace_bytes(8, 0) == 0
    assert L.haf_lowrank_workspace_bytes(130, 2) == 0 and L.haf_lowrank_workspace_bytes(8, 17) == 0
    for nn, rr in ((2, 1), (8, 3), (56, 8)):
        assert L.haf_lowrank_workspace_bytes(nn, rr) >= 48 * math.comb(nn + rr - 1, rr - 1)
    assert L.haf_lowrank_launch(None, 4, 2, 256, 256, 1 << 20, None) == _native.HAF_EINVAL
    assert L.haf_lowrank_launch(256, 5, 2, 256, 256, 1 << 20, None) == _native.HAF_EINVAL
    assert L.haf_lowrank_launch(256, 4, 0, 256, 256, 1 << 20, None) == _native.HAF_EINVAL
    assert L.haf_lowrank_launch(256, 4, 2, 256, 8, 1 << 20, None) == _native.HAF_EINVAL  # misaligned
    assert L.haf_lowrank_launch(256, 8, 3, 256, 256, 64, None) == _native.HAF_ESMALL
    assert L.haf_tune(16, 1 << 7, 1, ctypes.byref(r)) == _native.HAF_EINVAL


def test_precision_limits_match_the_header():
    """The Python constants of the FP32 mode are the header's."""
    import paper_1805_12498_gb300 as hg
    src = open(os.path.join(ROOT, "include", "hafnian_gb300.h")).read()
    max_n = int(re.search(r"#define HAF_FP32_MAX_N (\d+)", src).group(1))
    tol = float(re.search(r"#define HAF_FP32_REL_TOL ([0-9.e+-]+)", src).group(1))
    tol64 = float(re.search(r"#define HAF_FP64_REL_TOL ([0-9.e+-]+)", src).group(1))
    gate = float(re.search(r"#define HAF_FP32_MAX_REL_ERR ([0-9.e+-]+)", src).group(1))
    code = int(re.search(r"#define HAF_EACCURACY \((-\d+)\)", src).group(1))
    assert hg.HAF_FP32_MAX_N == max_n and hg.HAF_FP32_REL_TOL == tol
    assert hg.HAF_FP64_REL_TOL == tol64 and hg.HAF_FP32_MAX_REL_ERR == gate and hg._native.HAF_EACCURACY == code
    assert int(re.search(r"#define HAF_FLAG_FP32 \(1u << (\d+)\)", src).group(1)) == 2
    with pytest.raises(ValueError):
        hg._flags(precision="fp16")


def test_noalloc_binding_checks_arguments_without_gpu_work():
    """The Python form of haf_launch_noalloc passes its arguments through;
    the library rejects bad sizes and null pointers before any CUDA call."""
    import paper_1805_12498_gb300 as hg
    from paper_1805_12498_gb300 import _native
    for bad_n in (0, 7, 58):
        with pytest.raises(hg.HafError) as e:
            hg.haf_launch_noalloc(0, bad_n, 0)
        assert e.value.code == _native.HAF_EINVAL and "HAF_MAX_N" in str(e.value)
    with pytest.raises(hg.HafError) as e:
        hg.haf_launch_noalloc(0, 8, 0, loops=True)
    assert e.value.code == _native.HAF_EINVAL and "null pointer" in str(e.value)
