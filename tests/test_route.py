"""The arithmetic route of the GPU kernels, restated in numpy on the CPU and
checked against the binary128 oracle's literal trace-power formula.

The kernels obtain each summand f(Z) from a Hessenberg form H of
B = (X A)^{(Z)} (a unitary similarity), La Budde's recurrence for
det(I - lambda H) truncated at degree h, and the series
g = det(I - lambda H)^{-1/2}; for the loop hafnian the reduction starts
from b = X v^T (a first reflector maps b to beta e_0, so the moments
u_k = a H^{k-1} b live on growing supports), u_k past N follow from
Cayley-Hamilton, and f = [lambda^h] g exp(sum_k u_k lambda^k / 2).  The
oracle instead raises B to explicit powers for the traces (Sec. 3.3,
eq. poly).  Agreement of the two on random subsets pins the route itself,
independently of the CUDA code.  No GPU needed.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from paper_1805_12498_gb300 import inputs


def submatrix(A, mask, h):
    """B = (X A)^{(Z)} with A's diagonal removed, and v = diag(A^{(Z)})."""
    pairs = [p for p in range(h) if (mask >> p) & 1]
    idx = [2 * p + s for p in pairs for s in (0, 1)]
    S = A[np.ix_(idx, idx)].copy()
    v = np.diag(S).copy()
    np.fill_diagonal(S, 0)
    X = np.zeros_like(S)
    for t in range(0, len(idx), 2):
        X[t, t + 1] = X[t + 1, t] = 1
    return X @ S, v, X


def labudde(H, h):
    """Coefficients d_0..d_h of det(I - lambda H) for upper Hessenberg H by
    the recurrence on leading principal submatrices, truncated at degree h
    (in H's precision)."""
    N = H.shape[0]
    D = [np.zeros(h + 1, dtype=H.dtype) for _ in range(N + 1)]
    D[0][0] = 1
    for i in range(1, N + 1):
        # D_i = (1 - lambda H_{i-1,i-1}) D_{i-1}
        #       - sum_{m=1}^{i-1} c_{i,m} lambda^{m+1} D_{i-1-m}
        cur = D[i - 1].copy()
        cur[1:] -= H[i - 1, i - 1] * D[i - 1][:-1]
        prod = 1.0 + 0j
        for m in range(1, i):
            prod *= H[i - m, i - m - 1]
            c = H[i - 1 - m, i - 1] * prod
            if m + 1 <= h:
                cur[m + 1:] -= c * D[i - 1 - m][: h + 1 - (m + 1)]
        D[i] = cur
    return D[N]


def summand(A, mask, h, loops, bulk=np.complex128):
    """f(Z) by the kernels' route.  ``bulk`` is the precision of the gather,
    the reflectors, the Hessenberg form, La Budde and the loop moments;
    the series and the Cayley-Hamilton continuation run in complex128 on the
    widened coefficients (complex64 models the FP32-bulk mode)."""
    B, v, X = submatrix(A, mask, h)
    B, v, X = B.astype(bulk), v.astype(bulk), X.astype(bulk)
    N = B.shape[0]
    if N == 0:
        return 0.0
    if loops:
        # Krylov start: a reflector P = I - w w^H maps b = X v to beta e_0
        b = X @ v
        x0 = b[0]
        nrm = np.linalg.norm(b)
        ph = x0 / abs(x0) if abs(x0) > 0 else 1.0
        w = b.copy()
        w[0] += ph * nrm
        w = w / np.linalg.norm(w) * np.sqrt(2) if np.linalg.norm(w) > 0 else w
        P = np.eye(N, dtype=bulk) - np.outer(w, w.conj())
        B = P @ B @ P
        a = v @ P
        b = P @ b  # = -ph * nrm e_0
        H, Q = sl.hessenberg(B, calc_q=True)  # Q e_0 = e_0
        a = a @ Q
        b = Q.conj().T @ b
        eps = np.finfo(bulk).eps
        assert np.allclose(b[1:], 0, atol=1e4 * eps * max(1.0, nrm))
    else:
        H = sl.hessenberg(B)
    d = labudde(H, h).astype(np.complex128)
    # g = D^{-1/2}: k g_k = -sum_{j=1}^{min(k,N)} (k - j/2) d_j g_{k-j}
    g = np.zeros(h + 1, dtype=complex)
    g[0] = 1
    for k in range(1, h + 1):
        g[k] = -sum((k - j / 2) * d[j] * g[k - j] for j in range(1, min(k, N) + 1)) / k
    if not loops:
        return g[h]
    u = np.zeros(h + 1, dtype=complex)
    y = b.copy()  # supported on e_0
    for k in range(1, min(h, N) + 1):
        u[k] = complex(a @ y)  # widened, like the coefficients
        y = H @ y
    for k in range(N + 1, h + 1):  # Cayley-Hamilton: sum_j d_j u_{k-j} = 0
        u[k] = -sum(d[j] * u[k - j] for j in range(1, N + 1))
    e = np.zeros(h + 1, dtype=complex)
    e[0] = 1
    for k in range(1, h + 1):
        e[k] = sum(j * u[j] / 2 * e[k - j] for j in range(1, k + 1)) / k
    return sum(g[k] * e[h - k] for k in range(h + 1))


@pytest.mark.parametrize("n", [6, 10, 14])
@pytest.mark.parametrize("loops", [False, True])
def test_route_matches_the_trace_formula(n, loops):
    h = n // 2
    for A in (inputs.complex_gaussian_symmetric(n, 900 + n), inputs.real_gaussian_symmetric(n, 950 + n)):
        masks = inputs.random_masks(h, 24, seed=n + 7 * loops)
        masks = np.unique(np.concatenate([masks, np.array([(1 << h) - 1, 1], dtype=np.uint64)]))
        masks = masks[masks > 0]
        want = oracle.terms(A, loops, masks)
        got = np.array([summand(np.asarray(A, dtype=complex), int(m), h, loops) for m in masks])
        assert np.allclose(got, want, rtol=1e-9, atol=1e-12 * np.max(np.abs(want))), (n, loops)


def test_labudde_is_the_characteristic_polynomial():
    """Untruncated, the recurrence gives det(I - lambda H) exactly."""
    g = inputs.rng(5)
    M = g.standard_normal((7, 7)) + 1j * g.standard_normal((7, 7))
    H = sl.hessenberg(M)
    d = labudde(H, 7)
    # det(I - lambda H) = prod (1 - lambda mu_i): coefficients from the eigenvalues
    mu = np.linalg.eigvals(M)
    want = np.array([1.0 + 0j])
    for m in mu:
        want = np.convolve(want, [1.0, -m])
    assert np.allclose(d, want, atol=1e-10 * np.max(np.abs(want)))


@pytest.mark.parametrize("n", [16, 20])
@pytest.mark.parametrize("loops", [False, True])
def test_single_precision_bulk_route_error(n, loops):
    """The FP32-bulk arithmetic (complex64 bulk steps, complex128 series and
    sum) over every subset of an n = 16 or 20 matrix, against the oracle's
    full sum.  Its error relative to sum_Z |f(Z)| (about 1e-8 to 1.3e-7 on
    these inputs) is checked against the FP32 mode's stated per-unit error
    HAF_FP32_REL_TOL of the C header.  The same route in complex128 stays
    below 1e-12 (about 1e-16 here), inside the FP64 contract of 1e-10."""
    import paper_1805_12498_gb300 as hg
    h = n // 2
    A = np.asarray(inputs.complex_gaussian_symmetric(n, 960 + n), dtype=complex)
    want, scale = oracle.haf_formula(A, loops)
    masks = range(1, 1 << h)
    signs = [(-1) ** (h - bin(m).count("1")) for m in masks]
    for bulk, bound in ((np.complex64, hg.HAF_FP32_REL_TOL), (np.complex128, 1e-12)):
        got = sum(sg * summand(A, m, h, loops, bulk) for sg, m in zip(signs, masks))
        assert abs(got - want) <= bound * scale, (bulk.__name__, abs(got - want) / scale)
