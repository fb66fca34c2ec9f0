"""Autotuner (haf_tune, haf_tune_set, haf_batched_tune): every launch shape
computes the same hafnian; the tuner records the fastest shape and later
calls use it."""
import numpy as np
import pytest

import oracle
import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import inputs, tuning

pytestmark = pytest.mark.gpu

TOL = 1e-10


def test_tune_records_a_shape_and_results_stay_exact():
    A = inputs.complex_gaussian_symmetric(24, 17)
    want, scale = oracle.haf_formula(A)
    r = hg.tune(24, reps=1)
    assert r["warps_per_block"] in (4, 8, 16) and 1 <= r["chunks_per_warp"] <= 64
    assert r["candidates"] >= 4 and r["ms"] > 0 and r["ms"] <= r["ms_default"] * 1.0001
    got = hg.haf_info(A)
    assert abs(got.value - want) <= TOL * scale


@pytest.mark.parametrize("wpb,cpw", [(4, 2), (8, 16), (16, 4)])
def test_every_shape_gives_the_same_value(wpb, cpw):
    """Including two-launch plans: at n = 40 the largest tiles do not fit an
    8- or 16-warp slice and run in a second, 4-warp launch."""
    n = 40
    J = np.ones((n, n))
    hg.tune_set(n, wpb, cpw, real=True)
    r = hg.haf_info(J, real=True)
    exact = 1.0
    for k in range(1, n, 2):
        exact *= k
    assert abs(r.value.real - exact) <= TOL * r.abs_sum
    A = inputs.complex_gaussian_symmetric(n, 4)
    hg.tune_set(n, wpb, cpw)
    a = hg.haf_info(A)
    hg.tune_set(n, 4, 8)
    b = hg.haf_info(A)
    assert abs(a.value - b.value) <= 1e-13 * b.abs_sum
    tuning.load()  # back to the shipped table


def test_batched_tune_keeps_results():
    _, mats = inputs.gbs_batch(32, seed=12, n_min=4, n_max=18)
    r = hg.batched_tune(mats, reps=1)
    assert r["warps_per_block"] in (4, 8, 16) and r["candidates"] >= 4
    vals = hg.haf_batched(mats)
    for M, v in zip(mats, vals):
        s = hg.haf_info(M)
        assert abs(v - s.value) <= TOL * s.abs_sum


def test_shipped_table_covers_every_size():
    import json
    import os
    assert os.path.exists(tuning.TABLE_PATH)
    table = json.load(open(tuning.TABLE_PATH))
    sh = tuning.shapes(table)
    for flags in (0, hg.HAF_FLAG_REAL, hg.HAF_FLAG_FP32):
        for n in range(2, hg.HAF_MAX_N + 1, 2):
            wpb, cpw = sh[(flags, n)]
            assert wpb in (4, 8, 16) and 1 <= cpw <= 64
