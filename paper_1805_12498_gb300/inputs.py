"""Seeded synthetic inputs for the hafnian workloads.

This module only draws inputs; it holds none of the hafnian arithmetic.
It is the one module shared by the library's users (benchmark) and the
test-suite's oracle checks.  All draws use numpy's counter-based Philox
bit generator, so a (seed, shape) pair names the same matrix on every
machine.

Workload shapes (Sec. 4 lists the paper's benchmark graphs):
  * complete graph: all-ones matrix, haf = (n-1)!!, lhaf = T(n);
  * complete bipartite graph: [[0, W], [W^T, 0]] with W all-ones;
  * random complex symmetric matrices: A = (G + G^T)/2 with complex
    Gaussian G, re and im ~ N(0, 1/2) (the paper draws uniform entries;
    Gaussian entries are used here, which keeps |A_ij| ~ 1);
  * real symmetric variants with N(0, 1) entries;
  * Gaussian-boson-sampling (GBS) submatrices: B = U diag(tanh r) U^T for a
    Haar-random unitary U, with rows/columns repeated by a click pattern
    (Sec. 1 motivates the hafnian by GBS probabilities).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def complex_gaussian_symmetric(n: int, seed: int) -> np.ndarray:
    """A = (G + G^T)/2, G_ij = x + i y with x, y ~ N(0, 1/2) i.i.d."""
    g = rng(seed)
    s = np.sqrt(0.5)
    G = g.standard_normal((n, n)) * s + 1j * (g.standard_normal((n, n)) * s)
    return np.ascontiguousarray((G + G.T) / 2)


def real_gaussian_symmetric(n: int, seed: int) -> np.ndarray:
    """A = (G + G^T)/2 with G_ij ~ N(0, 1) i.i.d. (float64)."""
    g = rng(seed)
    G = g.standard_normal((n, n))
    return np.ascontiguousarray((G + G.T) / 2)


def all_ones(n: int, dtype=np.complex128) -> np.ndarray:
    return np.ones((n, n), dtype=dtype)


def bipartite(W: np.ndarray) -> np.ndarray:
    """[[0, W], [W^T, 0]] (eq. bipartite)."""
    W = np.asarray(W)
    k = W.shape[0]
    A = np.zeros((2 * k, 2 * k), dtype=np.result_type(W.dtype, np.complex128))
    A[:k, k:] = W
    A[k:, :k] = W.T
    return A


def haar_unitary(m: int, seed: int) -> np.ndarray:
    """Haar-random m x m unitary: QR of a complex Gaussian matrix with the
    phases of R's diagonal moved into Q (Mezzadri's construction)."""
    g = rng(seed)
    Z = (g.standard_normal((m, m)) + 1j * g.standard_normal((m, m))) / np.sqrt(2)
    Q, R = np.linalg.qr(Z)
    d = np.diag(R)
    return Q * (d / np.abs(d))


def gbs_kernel(modes: int = 32, r: float = 0.88, seed: int = 0) -> np.ndarray:
    """B = U diag(tanh r) U^T, complex symmetric, for Haar U."""
    U = haar_unitary(modes, seed)
    t = np.full(modes, np.tanh(r))
    return np.ascontiguousarray((U * t) @ U.T)


def repeat_submatrix(B: np.ndarray, counts) -> np.ndarray:
    """Submatrix that repeats row/column i of B counts[i] times."""
    idx = np.repeat(np.arange(B.shape[0]), np.asarray(counts, dtype=np.int64))
    return np.ascontiguousarray(B[np.ix_(idx, idx)])


def click_pattern(n_photons: int, modes: int, g: np.random.Generator) -> np.ndarray:
    """Each of n photons lands in a mode drawn uniformly; returns counts."""
    modes_hit = g.integers(0, modes, size=n_photons)
    return np.bincount(modes_hit, minlength=modes)


def gbs_batch(count: int, seed: int, modes: int = 32, r: float = 0.88,
              n_min: int = 8, n_max: int = 32):
    """``count`` GBS submatrices with n uniform on the even numbers in
    [n_min, n_max]; returns (kernel B, list of matrices)."""
    B = gbs_kernel(modes, r, seed)
    g = rng(seed + 1)
    evens = np.arange(n_min, n_max + 1, 2)
    mats = []
    for _ in range(count):
        n = int(g.choice(evens))
        mats.append(repeat_submatrix(B, click_pattern(n, modes, g)))
    return B, mats


def lowrank_gaussian_integer(n: int, r: int, seed: int, amp: int = 1):
    """G (n x r) with re, im uniform on {-amp..amp}; returns (G, A = G G^T).
    A is computed exactly in integers, so it is exact in float64."""
    g = rng(seed)
    gre = g.integers(-amp, amp + 1, size=(n, r))
    gim = g.integers(-amp, amp + 1, size=(n, r))
    Are = gre @ gre.T - gim @ gim.T
    Aim = gre @ gim.T + gim @ gre.T
    return gre + 1j * gim, (Are + 1j * Aim).astype(np.complex128)


def random_masks(h: int, count: int, seed: int) -> np.ndarray:
    """``count`` uniformly random subsets of the h pairs, as uint64 bitmasks."""
    g = rng(seed)
    if h == 0:
        return np.zeros(count, dtype=np.uint64)
    hi = g.integers(0, 1 << min(h, 62), size=count, dtype=np.uint64)
    return hi
