"""Write tests/golden/oracle_values.json: oracle values for the seeded
parity cases too slow to recompute inside the GPU test run.

Every number in the file comes from ``oracle`` (the binary128 CPU oracle)
applied to inputs from ``paper_1805_12498_gb300.inputs``; nothing here calls
the CUDA library.

    python tests/golden/make_golden.py [--missing-only]

``--missing-only`` keeps the stored cases whose parameters are unchanged and
computes only the others.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1805_12498_gb300 import inputs  # noqa: E402

sys.path.insert(0, HERE)
import cases  # noqa: E402

CASES = [
    # (name, n, seed, loops, real)
    ("cgauss28_haf", 28, 28, False, False),
    ("cgauss28_lhaf", 28, 28, True, False),
    ("rgauss28_haf", 28, 128, False, True),
    ("rgauss28_lhaf", 28, 128, True, True),
    ("cgauss32_haf", 32, 32, False, False),
    ("cgauss32_lhaf", 32, 32, True, False),
    ("cgauss36_haf", 36, 36, False, False),
    ("cgauss36_lhaf", 36, 36, True, False),
    ("rgauss32_haf", 32, 132, False, True),
    ("rgauss32_lhaf", 32, 132, True, True),
    ("rgauss36_haf", 36, 136, False, True),
    ("rgauss36_lhaf", 36, 136, True, True),
    ("cgauss40_haf", 40, 40, False, False),
    ("rgauss40_haf", 40, 140, False, True),
]


def recipe_cases():
    """(name, params, matrix, loops) of every stored case: the complex and
    real Gaussian sweep above, the GBS submatrices and the large requests of
    the server mix (tests/golden/cases.py)."""
    for name, n, seed, loops, real in CASES:
        A = (inputs.real_gaussian_symmetric(n, seed) if real
             else inputs.complex_gaussian_symmetric(n, seed))
        yield name, {"n": n, "seed": seed, "loops": loops, "real": real}, A, loops
    for name, n, seed, loops in cases.GBS_CASES:
        yield name, {"n": n, "seed": seed, "loops": loops, "real": False, "recipe": "gbs_submatrix"}, \
            cases.gbs_submatrix(n, seed), loops
    for k, M, loops in cases.server_mix_stored(11):
        yield f"server11_req{k}", {"n": M.shape[0], "seed": 11, "loops": loops, "real": False,
                                   "recipe": f"server_mix[{k}]"}, cases.pad_odd(M), loops


def main():
    out = {"source": "oracle.haf_formula (binary128), inputs.complex_gaussian_symmetric / "
                     "inputs.real_gaussian_symmetric with the listed seeds, and the recipes of "
                     "tests/golden/cases.py (GBS submatrices, the server mix)",
           "cases": []}
    stored = {}
    path = os.path.join(HERE, "oracle_values.json")
    if "--missing-only" in sys.argv and os.path.exists(path):
        with open(path) as f:
            stored = {c["name"]: c for c in json.load(f)["cases"]}
    for name, params, A, loops in recipe_cases():
        c = stored.get(name)
        if c and all(c.get(k) == v for k, v in params.items()):
            out["cases"].append(c)
            continue
        t = time.time()
        v, s = oracle.haf_formula(A, loops)
        out["cases"].append({"name": name, **params, "re": v.real, "im": v.imag, "abs_sum": s})
        print(name, v, s, f"{time.time() - t:.1f}s", flush=True)
        with open(path, "w") as f:
            json.dump(out | {"cases": out["cases"] + [c for nm, c in stored.items()
                                                      if nm not in {x["name"] for x in out["cases"]}]},
                      f, indent=1)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
