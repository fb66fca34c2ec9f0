"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself (the paper's printed worked examples, closed forms,
brute force, a textbook identity, exact integer arithmetic).  No GPU."""
import os
from math import comb

import numpy as np
import pytest

import oracle
from paper_1805_12498_gb300 import inputs

from golden import cases as golden_cases

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rel(a, b, scale):
    return abs(complex(a) - complex(b)) / max(scale, 1e-300)


# ---------------------------------------------------------------- Sec. 2 --
def _worked_expansions():
    out = {"haf": [], "lhaf": []}
    with open(os.path.join(GOLDEN, "worked_4x4.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            kind, rest = line.split(":")
            pairs = [tuple(int(x) for x in p.split(",")) for p in rest.split()]
            out[kind.strip()].append(pairs)
    return out


def test_worked_4x4_expansions_match_brute_force():
    """eq. hafB and the printed lhaf(B) sum (Sec. 2) against enumeration."""
    ex = _worked_expansions()
    assert len(ex["haf"]) == 3 and len(ex["lhaf"]) == 10  # |PMP(4)|, |SPM(4)|
    for seed in range(5):
        B = inputs.complex_gaussian_symmetric(4, 100 + seed)
        for kind, loops in (("haf", False), ("lhaf", True)):
            want = sum(np.prod([B[i, j] for i, j in m]) for m in ex[kind])
            got = oracle.haf_brute(B, loops)
            assert abs(got - want) <= 1e-15 * (1 + abs(want))
            got_f, _ = oracle.haf_formula(B, loops)
            assert abs(got_f - want) <= 1e-14 * (1 + abs(want))


@pytest.mark.parametrize("n", list(range(0, 17, 2)))
def test_brute_all_ones_is_double_factorial(n):
    """|PMP(n)| = (n-1)!! (eq. haf1)."""
    assert oracle.haf_brute(np.ones((n, n))) == oracle.double_factorial(n - 1)


@pytest.mark.parametrize("n", list(range(0, 13)))
def test_brute_all_ones_loops_is_telephone(n):
    """|SPM(n)| = T(n) (eq. haf2, App. A); odd n allowed for the loop case."""
    assert oracle.haf_brute(np.ones((n, n)), loops=True) == oracle.telephone(n)


def test_telephone_recurrence_matches_appendix_a_sum():
    for n in range(0, 41, 2):
        assert oracle.telephone(n) == oracle.telephone_appendix_a(n)
        assert oracle.telephone(n) == oracle.telephone_kummer(n)
    # small known values of the telephone numbers
    assert [oracle.telephone(k) for k in range(9)] == [1, 1, 2, 4, 10, 26, 76, 232, 764]


def test_brute_ignores_diagonal_and_lower_triangle():
    """haf depends only on the upper triangle (Sec. 2; App. C, haf(A+L))."""
    A = inputs.complex_gaussian_symmetric(10, 7)
    L = np.tril(inputs.complex_gaussian_symmetric(10, 8))
    assert abs(oracle.haf_brute(A) - oracle.haf_brute(A + L)) == 0


def test_brute_odd_sizes():
    """No perfect matching for odd n; lhaf(A) for odd n equals lhaf of A with
    an isolated vertex of loop weight 1 appended."""
    for n in (1, 3, 5, 7):
        A = inputs.complex_gaussian_symmetric(n, 11 + n)
        assert oracle.haf_brute(A) == 0
        Ap = np.zeros((n + 1, n + 1), dtype=complex)
        Ap[:n, :n] = A
        Ap[n, n] = 1
        assert abs(oracle.haf_brute(A, True) - oracle.haf_brute(Ap, True)) <= 1e-14 * (
            1 + abs(oracle.haf_brute(A, True)))


# ---------------------------------------------------------- Sec. 3.2-3.3 --
@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12, 14])
def test_formula_matches_brute_force_haf(n):
    A = inputs.complex_gaussian_symmetric(n, 1000 + n)
    want = oracle.haf_brute(A)
    got, s = oracle.haf_formula(A)
    assert _rel(got, want, s) <= 1e-25 or abs(got - want) <= 1e-13 * abs(want)


@pytest.mark.parametrize("n", [2, 4, 6, 8, 10, 12])
def test_formula_matches_brute_force_lhaf(n):
    A = inputs.complex_gaussian_symmetric(n, 2000 + n)
    want = oracle.haf_brute(A, True)
    got, s = oracle.haf_formula(A, True)
    assert abs(got - want) <= 1e-13 * max(abs(want), 1e-300)


@pytest.mark.parametrize("n", [4, 8, 12])
def test_formula_matches_brute_force_real(n):
    A = inputs.real_gaussian_symmetric(n, 3000 + n)
    for loops in (False, True):
        want = oracle.haf_brute(A, loops)
        got, _ = oracle.haf_formula(A, loops)
        assert abs(got - want) <= 1e-13 * max(abs(want), 1e-300)


def test_printed_loop_term_is_rejected_by_brute_force():
    """The loop term exactly as printed, v (X B)^{k-1} v^T / 2, disagrees
    with the definition; the oracle's reading u_k = v B^{k-1} X v^T agrees.
    (This is the test that pins the reading of the garbled formula.)"""
    for n in (2, 4, 6):
        A = inputs.complex_gaussian_symmetric(n, 4000 + n)
        want = oracle.haf_brute(A, True)
        good, _ = oracle.haf_formula(A, True, variant=0)
        bad, _ = oracle.haf_formula(A, True, variant=1)
        assert abs(good - want) <= 1e-13 * abs(want)
        assert abs(bad - want) > 1e-3 * abs(want)


@pytest.mark.parametrize("n", [2, 8, 16, 20])
def test_formula_all_ones(n):
    got, _ = oracle.haf_formula(np.ones((n, n)))
    assert got == oracle.double_factorial(n - 1)
    got, _ = oracle.haf_formula(np.ones((n, n)), True)
    assert abs(got - oracle.telephone(n)) <= 1e-20 * oracle.telephone(n) + 0.5


@pytest.mark.parametrize("n", [8, 16, 20])
def test_formula_rank_one_closed_forms(n):
    """A = x x^T with complex x: every perfect matching has weight prod x_i,
    so haf = (n-1)!! prod x_i (eq. haf1).  With the diagonal replaced by x,
    every single-pair matching has weight prod x_i too, so lhaf = T(n) prod x_i
    (eq. haf2).  Pins the formula with complex entries beyond brute force."""
    g = inputs.rng(7000 + n)
    x = (g.standard_normal(n) + 1j * g.standard_normal(n)) / np.sqrt(2)
    A = np.outer(x, x)
    p = np.prod(x)
    got, _ = oracle.haf_formula(A)
    want = oracle.double_factorial(n - 1) * p
    assert abs(got - want) <= 1e-13 * abs(want)
    np.fill_diagonal(A, x)
    got, _ = oracle.haf_formula(A, True)
    want = oracle.telephone(n) * p
    assert abs(got - want) <= 1e-13 * abs(want)


def test_formula_lhaf_of_a_diagonal_matrix():
    """Only the all-loops matching survives: lhaf(diag(d)) = prod d_i, and
    haf(diag(d)) = 0 (the loop series alone, Sec. 3.3)."""
    n = 20
    g = inputs.rng(7100)
    d = g.standard_normal(n) + 1j * g.standard_normal(n)
    got, _ = oracle.haf_formula(np.diag(d), True)
    assert abs(got - np.prod(d)) <= 1e-13 * abs(np.prod(d))
    got, _ = oracle.haf_formula(np.diag(d))
    assert got == 0


def test_formula_zero_size():
    assert oracle.haf_formula(np.zeros((0, 0)))[0] == 1


def test_formula_lhaf_equals_haf_for_zero_diagonal():
    """q(lambda, B, 0) = p(lambda, B) (Sec. 3.3)."""
    A = inputs.complex_gaussian_symmetric(12, 5)
    np.fill_diagonal(A, 0)
    a, _ = oracle.haf_formula(A)
    b, _ = oracle.haf_formula(A, True)
    assert abs(a - b) <= 1e-14 * abs(a)


def test_formula_scaling_laws():
    """haf(mu A) = mu^{n/2} haf(A); lhaf(sqrt(mu) A_diag + mu A_off) =
    mu^{n/2} lhaf(A) (eq. scaling)."""
    n, mu = 12, 1.7
    A = inputs.complex_gaussian_symmetric(n, 6)
    h0, _ = oracle.haf_formula(A)
    h1, _ = oracle.haf_formula(mu * A)
    assert abs(h1 - mu ** (n // 2) * h0) <= 1e-13 * abs(h1)
    D = np.diag(np.diag(A))
    l0, _ = oracle.haf_formula(A, True)
    l1, _ = oracle.haf_formula(np.sqrt(mu) * D + mu * (A - D), True)
    assert abs(l1 - mu ** (n // 2) * l0) <= 1e-13 * abs(l1)


def test_formula_permutation_invariance():
    """Any pairing of the vertices works (Sec. 3.2): haf(P A P^T) = haf(A)."""
    n = 14
    A = inputs.complex_gaussian_symmetric(n, 9)
    perm = inputs.rng(10).permutation(n)
    B = A[np.ix_(perm, perm)]
    for loops in (False, True):
        a, s = oracle.haf_formula(A, loops)
        b, _ = oracle.haf_formula(B, loops)
        assert abs(a - b) <= 1e-20 * s + 1e-13 * abs(a)


def test_formula_block_diagonal_factorises():
    A = inputs.complex_gaussian_symmetric(6, 21)
    C = inputs.complex_gaussian_symmetric(8, 22)
    M = np.zeros((14, 14), dtype=complex)
    M[:6, :6] = A
    M[6:, 6:] = C
    for loops in (False, True):
        want = oracle.haf_brute(A, loops) * oracle.haf_brute(C, loops)
        got, _ = oracle.haf_formula(M, loops)
        assert abs(got - want) <= 1e-13 * abs(want)


def test_formula_permuted_block_diagonal_n24():
    """haf(P (A + C) P^T) = haf(A) haf(C) for two random complex 12 x 12
    blocks under a random vertex permutation P (Sec. 2; any pairing works,
    Sec. 3.2), and the same for lhaf.  The permutation puts vertices of both
    blocks into the same pairs, so the subset sum does not factorise term by
    term; the expected value comes from brute force on each block.  This
    pins the formula on fully random complex input at n = 24."""
    A = inputs.complex_gaussian_symmetric(12, 23)
    C = inputs.complex_gaussian_symmetric(12, 24)
    M = np.zeros((24, 24), dtype=complex)
    M[:12, :12] = A
    M[12:, 12:] = C
    perm = inputs.rng(25).permutation(24)
    M = M[np.ix_(perm, perm)]
    for loops in (False, True):
        want = oracle.haf_brute(A, loops) * oracle.haf_brute(C, loops)
        got, s = oracle.haf_formula(M, loops)
        assert abs(got - want) <= 1e-14 * abs(want), (loops, got, want, s)


def test_terms_sum_to_formula():
    """The per-subset entry point gives the same summands (signed sum)."""
    n = 12
    h = n // 2
    A = inputs.complex_gaussian_symmetric(n, 31)
    masks = np.arange(1 << h, dtype=np.uint64)
    f = oracle.terms(A, False, masks)
    signs = np.array([(-1) ** (h - bin(int(z)).count("1")) for z in masks])
    got = np.sum(signs * f)
    want, s = oracle.haf_formula(A)
    assert abs(got - want) <= 1e-14 * s
    assert abs(np.sum(np.abs(f)) - s) <= 1e-12 * s


# ------------------------------------------------------- eq. bipartite ---
def test_ryser_matches_permutation_sum():
    for k in range(1, 7):
        W = inputs.complex_gaussian_symmetric(k, 40 + k) + 0.3j * np.eye(k)
        W = W + inputs.rng(50 + k).standard_normal((k, k))  # not symmetric
        want = oracle.permanent_by_permutations(W)
        assert abs(oracle.ryser(W) - want) <= 1e-13 * (1 + abs(want))


def test_ryser_all_ones_is_factorial():
    import math
    for k in range(0, 13):
        assert oracle.ryser(np.ones((k, k))) == math.factorial(k)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 7])
def test_bipartite_identity(k):
    """haf([[0, W], [W^T, 0]]) = per(W) (eq. bipartite)."""
    g = inputs.rng(60 + k)
    W = g.standard_normal((k, k)) + 1j * g.standard_normal((k, k))
    A = inputs.bipartite(W)
    want = oracle.ryser(W)
    got_b = oracle.haf_brute(A)
    got_f, s = oracle.haf_formula(A)
    assert abs(got_b - want) <= 1e-13 * (1 + abs(want))
    assert abs(got_f - want) <= 1e-12 * (1 + abs(want))


# ------------------------------------------------------------- App. C ----
@pytest.mark.parametrize("n,r", [(4, 2), (6, 2), (8, 3), (10, 2), (12, 3)])
def test_lowrank_exact_matches_brute_force(n, r):
    G, A = inputs.lowrank_gaussian_integer(n, r, seed=70 + n + r)
    re, im = oracle.haf_lowrank_exact(G)
    got = oracle.haf_brute(A)
    assert got == complex(re, im)


@pytest.mark.parametrize("n,r", [(16, 2), (20, 3)])
def test_lowrank_exact_matches_formula(n, r):
    G, A = inputs.lowrank_gaussian_integer(n, r, seed=80 + n + r)
    re, im = oracle.haf_lowrank_exact(G)
    got, s = oracle.haf_formula(A)
    assert abs(got - complex(re, im)) <= 1e-20 * s + 1e-12 * abs(complex(re, im))


def test_lowrank_exact_all_ones_rank_one():
    """J_n = g g^T with g = ones: haf = (n-1)!! at any size."""
    for n in (2, 10, 30, 56):
        re, im = oracle.haf_lowrank_exact(np.ones((n, 1)))
        assert (re, im) == (oracle.double_factorial(n - 1), 0)


def test_lowrank_monomial_count():
    """|E_{2n,r}| = C(n+r-1, r-1) even partitions (App. C)."""
    n2, r = 12, 3
    count = sum(1 for a in range(0, n2 + 1, 2) for b in range(0, n2 + 1 - a, 2)
                if (n2 - a - b) % 2 == 0)
    assert count == comb(n2 // 2 + r - 1, r - 1)


# ------------------------------------------------------ stored values ----
def test_stored_oracle_values_come_from_the_oracle():
    """tests/golden/oracle_values.json is written by make_golden.py, which
    calls only the oracle.  Recomputing its cheapest case (real n = 28, haf)
    reproduces the stored value and abs_sum; every case's inputs are the
    seeded generators' and its sizes are even and within the formula's range."""
    import json
    with open(os.path.join(GOLDEN, "oracle_values.json")) as f:
        cases = json.load(f)["cases"]
    names = [c["name"] for c in cases]
    assert len(set(names)) == len(names)
    for c in cases:
        ne = golden_cases.evaluated_size(c["n"], c["loops"])
        assert ne % 2 == 0 and 2 <= ne <= 48 and c["abs_sum"] > 0
    c = next(c for c in cases if c["name"] == "rgauss28_haf")
    A = inputs.real_gaussian_symmetric(c["n"], c["seed"])
    v, s = oracle.haf_formula(A, c["loops"])
    assert abs(v - complex(c["re"], c["im"])) <= 1e-15 * s
    assert abs(s - c["abs_sum"]) <= 1e-14 * s
