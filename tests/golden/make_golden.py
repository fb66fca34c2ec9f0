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


def main():
    out = {"source": "oracle.haf_formula (binary128), inputs.complex_gaussian_symmetric / "
                     "inputs.real_gaussian_symmetric with the listed seeds",
           "cases": []}
    stored = {}
    path = os.path.join(HERE, "oracle_values.json")
    if "--missing-only" in sys.argv and os.path.exists(path):
        with open(path) as f:
            stored = {c["name"]: c for c in json.load(f)["cases"]}
    for name, n, seed, loops, real in CASES:
        c = stored.get(name)
        if c and (c["n"], c["seed"], c["loops"], c["real"]) == (n, seed, loops, real):
            out["cases"].append(c)
            continue
        A = (inputs.real_gaussian_symmetric(n, seed) if real
             else inputs.complex_gaussian_symmetric(n, seed))
        t = time.time()
        v, s = oracle.haf_formula(A, loops)
        out["cases"].append({"name": name, "n": n, "seed": seed, "loops": loops, "real": real,
                             "re": v.real, "im": v.imag, "abs_sum": s})
        print(name, v, s, f"{time.time() - t:.1f}s", flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
