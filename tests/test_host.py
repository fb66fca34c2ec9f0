"""Host-side logic without a GPU: the seeded input generators (the recipe
of the paper's workloads), the launch-shape table's interpolation, and the
flag mapping of the Python front end."""
import numpy as np
import pytest

import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import _native, inputs, tuning


def test_generators_are_seeded_and_symmetric():
    a = inputs.complex_gaussian_symmetric(12, 5)
    b = inputs.complex_gaussian_symmetric(12, 5)
    c = inputs.complex_gaussian_symmetric(12, 6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert np.array_equal(a, a.T) and a.dtype == np.complex128
    r = inputs.real_gaussian_symmetric(10, 3)
    assert np.array_equal(r, r.T) and r.dtype == np.float64
    # entry scale: off-diagonal re, im ~ N(0, 1/4) after symmetrisation
    big = inputs.complex_gaussian_symmetric(400, 1)
    off = big[np.triu_indices(400, 1)]
    assert abs(np.var(off.real) - 0.25) < 0.01 and abs(np.var(off.imag) - 0.25) < 0.01


def test_gbs_kernel_recipe():
    U = inputs.haar_unitary(32, 7)
    assert np.allclose(U @ U.conj().T, np.eye(32), atol=1e-12)
    B = inputs.gbs_kernel(32, 0.88, 7)
    assert np.allclose(B, B.T, atol=1e-14)
    # B = U diag(tanh r) U^T: its singular values are all tanh r
    assert np.allclose(np.linalg.svd(B, compute_uv=False), np.tanh(0.88), atol=1e-12)
    g = inputs.rng(3)
    counts = inputs.click_pattern(20, 32, g)
    assert counts.sum() == 20 and counts.shape == (32,)
    M = inputs.repeat_submatrix(B, counts)
    assert M.shape == (20, 20) and np.allclose(M, M.T)
    _, mats = inputs.gbs_batch(64, seed=4, n_min=8, n_max=32)
    ns = [m.shape[0] for m in mats]
    assert all(8 <= n <= 32 and n % 2 == 0 for n in ns) and len(set(ns)) > 4


def test_haar_unitary_is_haar_distributed():
    """Mezzadri's construction: with the phases of R's diagonal moved into Q,
    every entry of a Haar unitary has mean 0 and E|U_ij|^2 = 1/m.  QR alone
    (LAPACK's sign convention) gives Re U_00 a mean near -0.28 at m = 4.
    Over 4000 fixed seeds the standard error of the mean is about 0.006."""
    u = np.array([inputs.haar_unitary(4, s)[0, 0] for s in range(4000)])
    assert abs(u.mean()) < 0.03
    assert abs(np.mean(np.abs(u) ** 2) - 0.25) < 0.02


def test_lowrank_and_mask_generators():
    G, A = inputs.lowrank_gaussian_integer(9, 3, seed=2)
    assert np.array_equal(A, G @ G.T)  # integer entries: exact in float64
    m = inputs.random_masks(20, 1000, seed=1)
    assert m.dtype == np.uint64 and int(m.max()) < (1 << 20)
    assert len(set(m.tolist())) > 900


def test_shape_table_takes_the_nearest_size_below():
    table = {"entries": [
        {"flags": 0, "n": 16, "warps_per_block": 16, "chunks_per_warp": 2},
        {"flags": 0, "n": 32, "warps_per_block": 8, "chunks_per_warp": 16},
        {"flags": 4, "n": 20, "warps_per_block": 16, "chunks_per_warp": 4},
    ]}
    sh = tuning.shapes(table)
    assert sh[(0, 2)] == (16, 2)      # below the smallest: the smallest
    assert sh[(0, 30)] == (16, 2)
    assert sh[(0, 32)] == (8, 16)
    assert sh[(0, 56)] == (8, 16)
    assert sh[(4, 48)] == (16, 4)
    assert all(n % 2 == 0 for (_, n) in sh) and len(sh) == 2 * (_native.HAF_MAX_N // 2)


def test_shipped_table_is_well_formed():
    import json
    t = json.load(open(tuning.TABLE_PATH))
    for e in t["entries"]:
        assert e["warps_per_block"] in (4, 8, 16) and 1 <= e["chunks_per_warp"] <= 64
        assert e["ms"] <= e["ms_default"] * 1.0001 or e["ms_default"] < 0


def test_flag_mapping():
    assert hg._flags() == 0
    assert hg._flags(loops=True) == _native.HAF_FLAG_LOOPS
    assert hg._flags(real=True, precision="fp32") == _native.HAF_FLAG_REAL | _native.HAF_FLAG_FP32
    with pytest.raises(ValueError):
        hg._flags(precision="fp64x")
