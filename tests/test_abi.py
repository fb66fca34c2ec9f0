"""The C-ABI library builds, loads and exports every function that
include/*.h declares.  No compute calls (this runs without a GPU)."""
import ctypes
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
                 "lhaf_c128_batched", "haf_launch", "haf_workspace_bytes", "haf_terms_c128"):
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
