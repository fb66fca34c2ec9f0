"""Seeded recipes of the parity cases whose oracle values are stored in
oracle_values.json.  This module only draws inputs (through
paper_1805_12498_gb300.inputs); it holds no hafnian arithmetic.  Both
make_golden.py (which calls only the oracle) and the GPU tests build their
matrices from here, so a stored value and the matrix it belongs to can
never drift apart.
"""
from __future__ import annotations

from paper_1805_12498_gb300 import inputs

# Sizes above this are too slow for the oracle at test time and are stored.
TEST_TIME_MAX_N = 24


def gbs_submatrix(n: int, seed: int):
    """A GBS-shaped n x n matrix: the rows/columns of a 32-mode kernel
    B = U diag(tanh 0.88) U^T repeated by a click pattern of n photons."""
    B = inputs.gbs_kernel(32, 0.88, seed)
    return inputs.repeat_submatrix(B, inputs.click_pattern(n, 32, inputs.rng(seed + 1)))


# (name, n, seed, loops): GBS submatrices at the large end of the batched
# workload's size range (n even in [8, 32]).
GBS_CASES = [
    ("gbs28_haf", 28, 2801, False),
    ("gbs28_lhaf", 28, 2801, True),
    ("gbs32_haf", 32, 3201, False),
    ("gbs32_lhaf", 32, 3201, True),
]


def server_mix(seed: int = 11):
    """The request mix of the server tests: 36 GBS submatrices with n drawn
    from {2, ..., 28} (a few odd sizes), haf/lhaf alternating, then one
    complex Gaussian n = 34 haf.  Returns a list of (matrix, loops)."""
    B = inputs.gbs_kernel(32, 0.88, seed)
    g = inputs.rng(seed + 1)
    reqs = []
    for k in range(36):
        n = int(g.choice([2, 6, 8, 10, 12, 16, 20, 24, 28])) + (1 if k % 9 == 4 else 0)
        M = inputs.repeat_submatrix(B, inputs.click_pattern(n, 32, g))
        reqs.append((M, bool(k % 2)))
    reqs.append((inputs.complex_gaussian_symmetric(34, seed + 2), False))
    return reqs


def evaluated_size(n: int, loops: bool) -> int:
    """Size the library evaluates: an odd lhaf is padded by one isolated
    looped vertex; an odd haf is 0 without any evaluation (size 0)."""
    if n % 2 == 0:
        return n
    return n + 1 if loops else 0


def server_mix_stored(seed: int = 11):
    """Indices and (matrix, loops) of the server-mix requests whose oracle
    value is stored (evaluated size above TEST_TIME_MAX_N)."""
    return [(k, M, loops) for k, (M, loops) in enumerate(server_mix(seed))
            if evaluated_size(M.shape[0], loops) > TEST_TIME_MAX_N]


def pad_odd(M):
    """An odd-size matrix with one isolated vertex of loop weight 1 appended
    (the odd-n loop-hafnian convention: such a vertex can only be matched to
    itself, so it multiplies lhaf by 1).  Even sizes are returned as given."""
    import numpy as np

    n = M.shape[0]
    if n % 2 == 0:
        return M
    P = np.zeros((n + 1, n + 1), dtype=np.complex128)
    P[:n, :n] = M
    P[n, n] = 1.0
    return P


def stored_case(name: str) -> dict:
    """The record of a stored oracle case (oracle_values.json)."""
    import json
    import os

    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")) as f:
        for c in json.load(f)["cases"]:
            if c["name"] == name:
                return c
    raise KeyError(name)


def stored(name: str):
    """(value, abs_sum) of a stored oracle case."""
    c = stored_case(name)
    return complex(c["re"], c["im"]), float(c["abs_sum"])


def case_matrix(c):
    """The input matrix of a stored case (a record of oracle_values.json),
    rebuilt from its recipe."""
    recipe = c.get("recipe")
    if recipe is None:
        return (inputs.real_gaussian_symmetric(c["n"], c["seed"]) if c["real"]
                else inputs.complex_gaussian_symmetric(c["n"], c["seed"]))
    if recipe == "gbs_submatrix":
        return gbs_submatrix(c["n"], c["seed"])
    if recipe.startswith("server_mix["):
        k = int(recipe[len("server_mix["):-1])
        return server_mix(c["seed"])[k][0]
    raise ValueError(f"unknown recipe {recipe}")
