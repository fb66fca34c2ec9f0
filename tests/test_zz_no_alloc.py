"""haf_launch_noalloc: the allocation-free entry point, for callers that may
not allocate device memory when they ask for a hafnian (memory pools that
own the device, callbacks that must not synchronise the device through
cudaMalloc/cudaFree, services with a fixed footprint).  Its scratch is one
static device array inside the library.

The test calls it through the C ABI twice in a row on the same stream (the
second call reuses the array the first one left behind) and compares both
results with the host entry point haf_c128 / lhaf_c128 within the
library's accuracy contract, |difference| <= 1e-10 * sum_Z |f(Z)|, and with
the binary128 oracle (at test time up to n = 24, stored sums above).
This file sorts last so that a run stopping at the first failure has run
every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import _native, inputs

from golden import cases as golden_cases

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _noalloc_fn():
    L = _native.lib()
    f = L.haf_launch_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _run(fn, A, flags, stream, dev, torch):
    n = A.shape[0]
    dA = torch.from_numpy(np.ascontiguousarray(A).view(np.float64).copy()).to(dev)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device=dev)
    rc = fn(dA.data_ptr(), n, flags, out.data_ptr(), stream.cuda_stream)
    assert rc == 0, _native.lib().haf_last_error()
    stream.synchronize()
    o = out.cpu().numpy()
    return complex(o[0] + o[2], o[1] + o[3]), float(o[4])


@pytest.mark.parametrize("n,loops", [(24, False), (22, True), (32, False)])
def test_noalloc_matches_host_entry_point_twice(n, loops):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    fn = _noalloc_fn()
    flags = _native.HAF_FLAG_LOOPS if loops else 0
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        A = inputs.complex_gaussian_symmetric(n, 4000 + 10 * n + call)
        ref = hg.haf_info(A, loops=loops)
        got, abs_sum = _run(fn, A, flags, stream, dev, torch)
        assert abs(got - ref.value) <= TOL * ref.abs_sum, (call, got, ref.value, ref.abs_sum)
        assert abs(abs_sum - ref.abs_sum) <= 1e-9 * ref.abs_sum
        if n <= 24:
            want, scale = oracle.haf_formula(A, loops)
            assert abs(got - want) <= TOL * scale, (call, got, want, scale)


@pytest.mark.parametrize("name,flags", [("cgauss40_haf", 0), ("cgauss36_lhaf", _native.HAF_FLAG_LOOPS),
                                        ("rgauss32_haf", _native.HAF_FLAG_REAL)])
def test_noalloc_against_stored_oracle_sums(name, flags):
    """The large and real cases of the header's range: complex n = 40 haf,
    complex n = 36 lhaf and a real n = 32 haf against the full binary128
    oracle sums, twice in a row (the second call reuses the array)."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    fn = _noalloc_fn()
    stream = torch.cuda.current_stream(dev)
    A = golden_cases.case_matrix(golden_cases.stored_case(name))
    want, scale = golden_cases.stored(name)
    for _ in range(2):
        got, abs_sum = _run(fn, A, flags, stream, dev, torch)
        assert abs(got - want) <= TOL * scale, (name, got, want, scale)
        assert abs(abs_sum - scale) <= 1e-8 * scale


def test_noalloc_rejects_sizes_beyond_the_limit():
    torch = pytest.importorskip("torch")
    fn = _noalloc_fn()
    dev = torch.device("cuda:0")
    dA = torch.zeros(2 * 58 * 58, dtype=torch.float64, device=dev)
    out = torch.zeros(5, dtype=torch.float64, device=dev)
    for bad_n in (58, 7, 0):
        rc = fn(dA.data_ptr(), bad_n, 0, out.data_ptr(), None)
        assert rc == _native.HAF_EINVAL
        assert b"HAF_MAX_N" in _native.lib().haf_last_error()
