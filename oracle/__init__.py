"""CPU oracle for the hafnian and the loop hafnian.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The
library (``paper_1805_12498_gb300``) never imports, links or runs it, and
shares no code with it.

What it provides (each function cites the passage it restates):

* ``haf_brute(A, loops)`` -- the definitions of Sec. 2: the sum over the
  perfect matchings PMP(n) (eq. hafA) or over the single-pair matchings
  SPM(n) (lhaf definition), accumulated in binary128.
* ``haf_formula(A, loops)`` -- the signed subset sum of Sec. 3.2 (eq. main)
  with each summand taken from the trace generating function of Sec. 3.3
  (eq. poly for haf, the q(lambda, B, v) function for lhaf), traces from
  explicit matrix powers, in binary128.
* ``terms(A, loops, masks)`` -- individual summands f(Z) of the same
  formula, for sampling large n.
* ``ryser(W)`` -- Ryser's permanent, for eq. bipartite.
* ``haf_lowrank_exact(G)`` -- App. C: the exact hafnian of G G^T for an
  integer (Gaussian-integer) n x r matrix G, in Python integers.
* ``double_factorial``, ``telephone`` -- the counts of eq. haf1 / eq. haf2
  (App. A), the hafnian and loop hafnian of the all-ones matrix.

Parity: every function above is pinned by tests in tests/test_oracle.py
(brute force against the worked 4x4 expansions of Sec. 2 and the closed
forms; the formula against brute force; Ryser against a permutation sum;
the low-rank evaluator against brute force).
"""
from __future__ import annotations

import ctypes
import os
from fractions import Fraction
from itertools import permutations
from math import comb

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_haf_brute.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_haf_brute.restype = ctypes.c_int
        lib.oracle_terms.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_uint64), ctypes.c_int64,
                                     ctypes.c_int, dp]
        lib.oracle_terms.restype = ctypes.c_int
        lib.oracle_haf_formula.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, dp, dp]
        lib.oracle_haf_formula.restype = ctypes.c_int
        lib.oracle_ryser.argtypes = [dp, ctypes.c_int, dp]
        lib.oracle_ryser.restype = ctypes.c_int
        _lib = lib
    return _lib


def _as_c128(A) -> np.ndarray:
    A = np.ascontiguousarray(np.asarray(A, dtype=np.complex128))
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    return A


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dd_to_complex(o) -> complex:
    return complex(o[0] + o[2], o[1] + o[3])


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def haf_brute(A, loops: bool = False) -> complex:
    """haf(A) or lhaf(A) by enumerating matchings (Sec. 2, eq. hafA; lhaf
    definition).  Reads the upper triangle (and the diagonal for lhaf).
    n <= 24; practical up to n = 16 (haf) / 14 (lhaf)."""
    A = _as_c128(A)
    out = np.zeros(4)
    rc = _load().oracle_haf_brute(_dp(A), A.shape[0], int(bool(loops)), _dp(out))
    if rc != 0:
        raise ValueError("oracle_haf_brute rejected the input")
    return _dd_to_complex(out)


def haf_formula(A, loops: bool = False, nthreads: int | None = None,
                variant: int = 0) -> tuple[complex, float]:
    """(value, sum_Z |f(Z)|) of the signed subset sum of eq. main with
    summands from eq. poly / q(lambda, B, v) (Sec. 3.2-3.3), binary128.
    ``variant=1`` uses the loop term exactly as printed (known to be wrong;
    kept so a test can show the pins reject it).  Even n <= 48."""
    A = _as_c128(A)
    out = np.zeros(4)
    s = np.zeros(1)
    rc = _load().oracle_haf_formula(_dp(A), A.shape[0], int(bool(loops)), int(variant),
                                    int(nthreads or default_threads()), _dp(out), _dp(s))
    if rc != 0:
        raise ValueError("oracle_haf_formula rejected the input")
    return _dd_to_complex(out), float(s[0])


def terms(A, loops: bool, masks, nthreads: int | None = None, variant: int = 0) -> np.ndarray:
    """Unsigned summands f(Z) for the subsets Z given as bitmasks over the
    n/2 pairs (bit i set <=> pair (2i, 2i+1) in Z).  Returns complex128."""
    A = _as_c128(A)
    masks = np.ascontiguousarray(np.asarray(masks, dtype=np.uint64))
    out = np.zeros((masks.size, 4))
    rc = _load().oracle_terms(_dp(A), A.shape[0], int(bool(loops)), int(variant),
                              masks.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                              masks.size, int(nthreads or default_threads()), _dp(out))
    if rc != 0:
        raise ValueError("oracle_terms rejected the input")
    return (out[:, 0] + out[:, 2]) + 1j * (out[:, 1] + out[:, 3])


def ryser(W) -> complex:
    """per(W) by Ryser's inclusion-exclusion formula (cited in Sec. 1), k <= 20."""
    W = _as_c128(W)
    out = np.zeros(4)
    rc = _load().oracle_ryser(_dp(W), W.shape[0], _dp(out))
    if rc != 0:
        raise ValueError("oracle_ryser rejected the input")
    return _dd_to_complex(out)


def permanent_by_permutations(W) -> complex:
    """per(W) = sum over permutations of prod W[i, s(i)]; tiny k only."""
    W = np.asarray(W, dtype=np.complex128)
    k = W.shape[0]
    total = 0j
    for s in permutations(range(k)):
        p = 1 + 0j
        for i in range(k):
            p *= W[i, s[i]]
        total += p
    return total


def double_factorial(a: int) -> int:
    """a!! = a (a-2) (a-4) ...; 1 for a <= 0 (App. C convention)."""
    r = 1
    while a > 0:
        r *= a
        a -= 2
    return r


def telephone(n: int) -> int:
    """T(n): the number of single-pair matchings of n vertices (eq. haf2),
    by the recurrence T(n) = T(n-1) + (n-1) T(n-2) (vertex n-1 either loops
    or pairs with one of the other n-1 vertices); tests tie it to the two
    App. A forms below."""
    t = [1, 1]
    for k in range(2, n + 1):
        t.append(t[k - 1] + (k - 1) * t[k - 2])
    return t[n]


def telephone_appendix_a(n: int) -> int:
    """The App. A sum for even n: breaking j pairs of each of the (n-1)!!
    perfect matchings in C(n/2, j) ways reaches each pattern with 2j loops
    (2j-1)!! times, so T(n) = sum_j (n-1)!! C(n/2, j) / (2j-1)!!.
    Reading: the sum is printed with (j-1)!! in the denominator, which
    gives 12 instead of T(4) = 10; the Kummer form printed on the next line,
    (n-1)!! M(-n/2, 1/2, -1/2), expands term by term to (2j-1)!!, which is
    the divisor used here (see ``telephone_kummer``)."""
    assert n % 2 == 0
    total = Fraction(0)
    for j in range(0, n // 2 + 1):
        total += Fraction(double_factorial(n - 1) * comb(n // 2, j), double_factorial(2 * j - 1))
    assert total.denominator == 1
    return int(total)


def telephone_kummer(n: int) -> int:
    """(n-1)!! M(-n/2, 1/2, -1/2) for even n, with Kummer's series
    M(a, b, z) = sum_k (a)_k z^k / ((b)_k k!) summed exactly (App. A)."""
    assert n % 2 == 0
    a, b, z = Fraction(-n, 2), Fraction(1, 2), Fraction(-1, 2)
    term, total, k = Fraction(1), Fraction(0), 0
    while term != 0:
        total += term
        term = term * (a + k) * z / ((b + k) * (k + 1))
        k += 1
    val = total * double_factorial(n - 1)
    assert val.denominator == 1
    return int(val)


def haf_lowrank_exact(G) -> tuple[int, int]:
    """Exact haf(G G^T) for an n x r matrix G of Gaussian integers (App. C).

    Expands q(x_1..x_r) = prod_i sum_j g_ij x_j (eq. q) as a polynomial with
    Gaussian-integer coefficients, then sums lambda_e prod_i (e_i - 1)!! over
    the even exponent vectors e.  The diagonal of G G^T plays no role (haf
    depends only on the upper triangle).  Returns (re, im) as Python ints.
    G is given as two integer arrays (re, im) or a complex array with
    integral parts."""
    G = np.asarray(G)
    n, r = G.shape
    gre = [[int(round(float(np.real(G[i, j])))) for j in range(r)] for i in range(n)]
    gim = [[int(round(float(np.imag(G[i, j])))) for j in range(r)] for i in range(n)]
    # poly: dict exponent-tuple -> (re, im)
    poly = {tuple([0] * r): (1, 0)}
    for i in range(n):
        nxt = {}
        for e, (pr, pi) in poly.items():
            for j in range(r):
                a, b = gre[i][j], gim[i][j]
                if a == 0 and b == 0:
                    continue
                e2 = list(e)
                e2[j] += 1
                e2 = tuple(e2)
                cr, ci = nxt.get(e2, (0, 0))
                nxt[e2] = (cr + pr * a - pi * b, ci + pr * b + pi * a)
        poly = nxt
    tr, ti = 0, 0
    for e, (pr, pi) in poly.items():
        if all(x % 2 == 0 for x in e):
            w = 1
            for x in e:
                w *= double_factorial(x - 1)
            tr += pr * w
            ti += pi * w
    return tr, ti
