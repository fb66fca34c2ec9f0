"""The usage example of the Python front end (as documented) runs and its
results agree with each other and with the closed forms they imply."""
import numpy as np
import pytest

import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_documented_usage():
    A = inputs.complex_gaussian_symmetric(40, seed=1)
    r = hg.haf_info(A)
    assert r.abs_sum > 0 and r.subsets == 2 ** 20 - 1
    l = hg.lhaf(A)
    with pytest.raises(hg.HafAccuracyError) as e:  # n = 40 cancels too much for FP32 bulk
        hg.haf(A, precision="fp32")
    assert abs(e.value.result.value - r.value) <= hg.HAF_FP32_REL_TOL * r.abs_sum
    S = A[:8, :8]
    f = hg.haf(S, precision="fp32")  # little cancellation at n = 8: admitted
    assert abs(f - hg.haf(S)) <= hg.HAF_FP32_MAX_REL_ERR * abs(hg.haf(S))
    vals = hg.haf_batched([A[:8, :8], A[:12, :12]])
    assert abs(vals[0] - hg.haf(A[:8, :8])) <= 1e-10 * hg.haf_info(A[:8, :8]).abs_sum
    with hg.Server() as srv:
        t = srv.submit(A, loops=True)
        v = srv.poll(t, timeout_s=120).value
    assert abs(v - l) <= 1e-10 * hg.haf_info(A, loops=True).abs_sum
    G, M = inputs.lowrank_gaussian_integer(56, 4, seed=2)
    lr = hg.haf_lowrank(G)
    assert np.isfinite(lr.value) and lr.abs_sum > 0
    rec = hg.haf_part(A, 0, 2)
    val, scale = hg.combine([rec, hg.haf_part(A, 1, 2)])
    assert abs(val - r.value) <= 1e-10 * r.abs_sum and scale == pytest.approx(r.abs_sum, rel=1e-12)
    shape = hg.tune(24)
    assert shape["warps_per_block"] in (4, 8, 16)
