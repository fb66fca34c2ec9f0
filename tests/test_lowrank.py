"""Low-rank hafnian on the GPU (App. C, haf_lowrank_c128): the expansion of
q(x) = prod_i sum_j g_ij x_j and the even-coefficient sum, against the
exact oracle (Python integers) and against the subset-sum path."""
import math

import numpy as np
import pytest

import oracle
import paper_1805_12498_gb300 as hg
from paper_1805_12498_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _close(got, want, scale):
    return abs(got - want) <= TOL * max(scale, 1e-300)


@pytest.mark.parametrize("n,r", [(2, 1), (4, 2), (8, 2), (12, 3), (16, 4), (24, 3), (32, 2), (40, 3),
                                 (48, 4), (56, 3), (64, 3), (96, 2)])
def test_lowrank_against_exact_oracle(n, r):
    G, A = inputs.lowrank_gaussian_integer(n, r, seed=7 * n + r)
    re, im = oracle.haf_lowrank_exact(G)
    got = hg.haf_lowrank(G)
    assert _close(got.value, complex(re, im), got.abs_sum), (n, r, got.value, re, im, got.abs_sum)
    assert got.subsets == math.comb(n + r - 1, r - 1)


@pytest.mark.parametrize("n,r", [(16, 3), (24, 5), (28, 8)])
def test_lowrank_against_subset_sum(n, r):
    """A complex Gaussian G: both algorithms of the library agree."""
    g = inputs.rng(100 + n + r)
    G = (g.normal(size=(n, r)) + 1j * g.normal(size=(n, r))) / np.sqrt(2 * r)
    a = hg.haf_lowrank(G)
    b = hg.haf_info(G @ G.T)
    assert _close(a.value, b.value, max(a.abs_sum, b.abs_sum)), (a.value, b.value)


def test_lowrank_edge_cases():
    assert hg.haf_lowrank(np.zeros((0, 2))).value == 1
    assert hg.haf_lowrank(np.ones((5, 2))).value == 0
    # rank one: haf(g g^T) = (n-1)!! prod_i g_i
    g = np.array([1.0, 2.0, -1.5, 0.5, 3.0, 1j])
    got = hg.haf_lowrank(g[:, None]).value
    want = 15 * np.prod(g)
    assert abs(got - want) <= 1e-12 * abs(want)
    # the diagonal and lower triangle of G G^T do not matter: a lower
    # triangular change of A = G G^T keeps the value (App. C)
    G, A = inputs.lowrank_gaussian_integer(10, 2, seed=3)
    L = np.tril(inputs.complex_gaussian_symmetric(10, 4))
    assert _close(hg.haf_info(A + L).value, hg.haf_lowrank(G).value, hg.haf_lowrank(G).abs_sum)


def test_lowrank_rejects_bad_sizes():
    with pytest.raises(hg.HafError):
        hg.haf_lowrank(np.ones((130, 2)))
    with pytest.raises(hg.HafError):
        hg.haf_lowrank(np.ones((8, 17)))


def _device_launch(G):
    """haf_lowrank_launch on device memory (torch tensors, current stream):
    the 5-double record {re_hi, im_hi, re_lo, im_lo, abs_sum}."""
    import torch
    n, r = G.shape
    dG = torch.from_numpy(np.ascontiguousarray(G, dtype=np.complex128).view(np.float64).copy()).cuda()
    ws = hg.lowrank_workspace_bytes(n, r)
    work = torch.empty(ws // 8 + 64, dtype=torch.float64, device="cuda")
    wptr = (work.data_ptr() + 255) // 256 * 256
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    hg.haf_lowrank_launch(dG.data_ptr(), n, r, out.data_ptr(), wptr, ws, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    rec = out.cpu().numpy()
    del work
    return rec


@pytest.mark.parametrize("n,r", [(2, 1), (12, 8), (24, 5), (40, 3)])
def test_lowrank_launch_on_device_memory(n, r):
    """The device-pointer form gives the host form's record bit for bit, and
    the exact value (integer G, Python-integer oracle)."""
    pytest.importorskip("torch")
    G, A = inputs.lowrank_gaussian_integer(n, r, seed=11 * n + r)
    rec = _device_launch(G)
    host = hg.haf_lowrank(G)
    assert complex(rec[0] + rec[2], rec[1] + rec[3]) == host.value and rec[4] == host.abs_sum
    re, im = oracle.haf_lowrank_exact(G)
    assert _close(host.value, complex(re, im), host.abs_sum), (n, r, host.value, re, im)


def test_lowrank_closed_form_at_n56_r8():
    """The benchmark size, n = 56 and r = 8 (5.5e8 monomials at degree 56):
    G_ij = g_i w_j, so G G^T = (sum_j w_j^2) g g^T and haf(G G^T) =
    (sum_j w_j^2)^(n/2) (n-1)!! prod_i g_i, while every coefficient of the
    expansion is nonzero and distinct: lambda_e = prod_i g_i * multinomial(n;
    e) * prod_j w_j^e_j.  With w_j > 0 the |g| expansion gives the modulus
    of the same value."""
    n, r = 56, 8
    g = inputs.rng(5608)
    gi = np.exp(1j * g.uniform(0, 2 * np.pi, size=n)) * g.uniform(0.8, 1.25, size=n)
    w = 1.0 + np.arange(r) / r
    G = np.outer(gi, w)
    dfact = float(math.prod(range(n - 1, 0, -2)))
    want = float(np.sum(w ** 2)) ** (n // 2) * dfact * np.prod(gi)
    got = hg.haf_lowrank(G)
    assert abs(got.value - want) <= 1e-12 * abs(want), (got.value, want)
    assert abs(got.abs_sum - abs(want)) <= 1e-12 * abs(want), (got.abs_sum, abs(want))
    assert got.subsets == math.comb(n + r - 1, r - 1)
