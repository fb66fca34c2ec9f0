"""FP32-bulk precision mode (HAF_FLAG_FP32): single-precision gather,
Householder reduction, loop moments and La Budde recurrence, FP64 series
and double-double subset sum.  Its error is stated relative to
abs_sum = sum_Z |f(Z)| (HAF_FP32_REL_TOL) and checked against the oracle
(small n) and against the FP64 path (which the oracle pins) at larger n.
Because the subset sum cancels, a whole-matrix FP32-bulk call is refused
(HAF_EACCURACY) when HAF_FP32_REL_TOL * abs_sum / |value| exceeds
HAF_FP32_MAX_REL_ERR; the tests of the error itself read the value that a
refused call still writes."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import inputs

from golden import cases as golden_cases

pytestmark = pytest.mark.gpu

TOL32 = hg.HAF_FP32_REL_TOL


def _fp32(A, loops=False, real=None):
    """The FP32-bulk result and report, whether the accuracy gate admits it
    or refuses it (a refused call still writes them)."""
    try:
        return hg.haf_info(A, loops, real=real, precision="fp32")
    except hg.HafAccuracyError as e:
        return e.result


def _gbs(n, seed):
    B = inputs.gbs_kernel(32, 0.88, seed)
    return inputs.repeat_submatrix(B, inputs.click_pattern(n, 32, inputs.rng(seed + 7)))


@pytest.mark.parametrize("n", [4, 8, 12, 16])
@pytest.mark.parametrize("loops", [False, True])
def test_fp32_against_oracle_small(n, loops):
    for A in (inputs.complex_gaussian_symmetric(n, 70 + n), _gbs(n, 80 + n)):
        want, scale = oracle.haf_formula(A, loops)
        got = _fp32(A, loops)
        assert abs(got.value - want) <= TOL32 * scale, (n, loops, got.value, want, scale)
        assert got.abs_sum == pytest.approx(scale, rel=1e-4)


@pytest.mark.parametrize("loops", [False, True])
def test_fp32_real_against_oracle(loops):
    A = inputs.real_gaussian_symmetric(14, 91)
    want, scale = oracle.haf_formula(A, loops)
    got = _fp32(A, loops, real=True)
    assert abs(got.value - want) <= TOL32 * scale


@pytest.mark.parametrize("n", [24, 32, 40])
def test_fp32_against_fp64(n):
    for A in (inputs.complex_gaussian_symmetric(n, 1000 + n), _gbs(n, 2000 + n)):
        for loops in (False, True):
            a = hg.haf_info(A, loops)
            b = _fp32(A, loops)
            assert abs(a.value - b.value) <= TOL32 * a.abs_sum, (n, loops)
            assert b.abs_sum == pytest.approx(a.abs_sum, rel=1e-4)


def test_fp32_against_stored_oracle_sums():
    """The FP32 mode against the full binary128 oracle sums that the FP64
    parity tests use (tests/golden/oracle_values.json: n = 28-40, complex
    and real, haf and lhaf), within the stated HAF_FP32_REL_TOL * sum |f|."""
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_values.json")
    with open(path) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        A = golden_cases.case_matrix(c)
        got = _fp32(A, c["loops"], real=c["real"])
        want = complex(c["re"], c["im"])
        assert abs(got.value - want) <= TOL32 * c["abs_sum"], (c["name"], got.value, want, c["abs_sum"])
        assert got.abs_sum == pytest.approx(c["abs_sum"], rel=1e-4), c["name"]


def test_fp32_terms_at_n48_against_oracle():
    """Sampled summands at the benchmark size against the binary128 oracle."""
    A = inputs.complex_gaussian_symmetric(48, 48)
    masks = inputs.random_masks(24, 48, seed=9)
    for loops in (False, True):
        want = oracle.terms(A, loops, masks)
        got = hg.haf_terms(A, masks, loops, precision="fp32")
        rel = np.abs(got - want) / np.abs(want)
        assert np.median(rel) <= 1e-4 and rel.max() <= 1e-1, (loops, np.median(rel), rel.max())
        f64 = hg.haf_terms(A, masks, loops)
        assert np.max(np.abs(f64 - want) / np.abs(want)) <= 1e-9


def test_fp32_batched_and_launch_forms():
    torch = pytest.importorskip("torch")
    _, mats = inputs.gbs_batch(24, seed=3, n_min=4, n_max=20)
    try:
        vals = hg.haf_batched(mats, precision="fp32")
    except hg.HafAccuracyError as e:  # some n = 14-20 matrices cancel too much
        vals = e.result[0]
    for M, v in zip(mats, vals):
        s = _fp32(M)
        assert abs(v - s.value) <= 1e-12 * s.abs_sum
    n = 20
    A = inputs.complex_gaussian_symmetric(n, 5)
    dev = torch.device("cuda:0")
    dA = torch.from_numpy(np.ascontiguousarray(A).view(np.float64)).to(dev)
    ws = hg.workspace_bytes(n, precision="fp32")
    work = torch.empty(ws // 8 + 64, dtype=torch.float64, device=dev)
    wptr = (work.data_ptr() + 255) // 256 * 256
    out = torch.zeros(5, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream()
    hg.haf_launch(dA.data_ptr(), n, out.data_ptr(), wptr, ws, st.cuda_stream, precision="fp32")
    st.synchronize()
    o = out.cpu().numpy()
    r = _fp32(A)
    assert complex(o[0] + o[2], o[1] + o[3]) == r.value


def test_fp32_mode_flags_and_limits():
    A = inputs.complex_gaussian_symmetric(8, 1)
    # the server and the no-alloc path stay FP64; unknown precision is rejected
    with pytest.raises(ValueError):
        hg.haf_info(A, precision="bf16")
    if hg.HAF_FP32_MAX_N < hg.HAF_MAX_N:
        B = inputs.complex_gaussian_symmetric(hg.HAF_FP32_MAX_N + 2, 1)
        with pytest.raises(hg.HafError):
            hg.haf_info(B, precision="fp32")


def test_fp32_accuracy_gate_admits_and_refuses():
    """The value-relative gate: a call is admitted exactly when the estimate
    HAF_FP32_REL_TOL * abs_sum / |value| is within HAF_FP32_MAX_REL_ERR, and
    then its error against the oracle is within that bound; the complex
    Gaussian n = 40 hafnian (stored oracle sum), whose FP32-bulk value has
    no correct digit, is refused."""
    admitted = 0
    for n in (4, 6, 8, 10, 12):
        for A in (np.ones((n, n), dtype=complex), inputs.complex_gaussian_symmetric(n, 300 + n),
                  _gbs(n, 310 + n)):
            want, scale = oracle.haf_formula(A)
            est = TOL32 * scale / abs(want)
            if est <= hg.HAF_FP32_MAX_REL_ERR:
                r = hg.haf_info(A, precision="fp32")
                assert r.precision_mode == 1 and r.rel_err_bound <= hg.HAF_FP32_MAX_REL_ERR
                assert abs(r.value - want) <= r.rel_err_bound * abs(want), (n, r.value, want)
                admitted += 1
            elif est > 2 * hg.HAF_FP32_MAX_REL_ERR:  # clear of the boundary
                with pytest.raises(hg.HafAccuracyError):
                    hg.haf_info(A, precision="fp32")
    assert admitted >= 8
    A = golden_cases.case_matrix({"n": 40, "seed": 40, "real": False})
    want, scale = golden_cases.stored("cgauss40_haf")
    with pytest.raises(hg.HafAccuracyError) as e:
        hg.haf_info(A, precision="fp32")
    r = e.value.result
    assert e.value.code == hg._native.HAF_EACCURACY and r.precision_mode == 1
    assert r.rel_err_bound > 1 and abs(r.value - want) > hg.HAF_FP32_MAX_REL_ERR * abs(want)
    assert abs(r.value - want) <= TOL32 * scale  # still within the stated error per unit of abs_sum
    # FP64 reports its own estimate and is never gated
    r64 = hg.haf_info(A)
    assert r64.precision_mode == 0 and abs(r64.value - want) <= r64.rel_err_bound * abs(want)
