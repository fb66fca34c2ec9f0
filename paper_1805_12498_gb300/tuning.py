"""Launch-shape table for GB300, written by the library's autotuner.

    python -m paper_1805_12498_gb300.tuning [--out PATH]   # on a GB300: regenerate

The autotuner (C ABI haf_tune) times every feasible launch shape of one
hafnian -- warps per CTA (4, 8 or 16; the shared-memory slice per warp,
hence the lanes per subset and the subsets per CTA, follow from it) and the
chunk granularity -- and keeps the fastest.  ``generate`` runs it over a
grid of sizes and kernel kinds and writes the shapes to a JSON table;
``load`` installs a table into the library (haf_tune_set) for every even n,
taking for each n the shape tuned at the largest tabulated size <= n.  The
Python entry points load the shipped table once, before their first GPU
call.  The shapes only steer scheduling: every shape computes the same sum
(the chunking, hence the last bits of the double-double sum, differ).
"""
from __future__ import annotations

import argparse
import json
import os

from . import _native

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_gb300.json")

# (kind name, flags, sizes tuned)
GRID = (
    ("c128", 0, (8, 12, 16, 20, 24, 28, 32, 36, 40, 44, 48)),
    ("f64", _native.HAF_FLAG_REAL, (16, 24, 32, 40, 48)),
    ("c64", _native.HAF_FLAG_FP32, (16, 20, 24, 28, 32, 36, 40, 44, 48, 52)),
)

_loaded = False


def generate(path: str = TABLE_PATH, reps: int = 1, grid=GRID) -> dict:
    """Run the autotuner over `grid` on the current GPU and write the table."""
    import ctypes

    L = _native.lib()
    entries = []
    for name, flags, sizes in grid:
        for n in sizes:
            r = _native.TuneResult()
            _native.check(L.haf_tune(n, flags, reps, ctypes.byref(r)))
            entries.append({"kind": name, "flags": flags, "n": n, "warps_per_block": r.warps_per_block,
                            "chunks_per_warp": r.chunks_per_warp, "ms": r.ms, "ms_default": r.ms_default,
                            "candidates": r.candidates})
            print(json.dumps(entries[-1]), flush=True)
    table = {"what": "fastest launch shape per (kernel kind, n) from haf_tune, one GB300",
             "reps": reps, "entries": entries}
    with open(path, "w") as f:
        json.dump(table, f, indent=1)
    return table


def shapes(table: dict) -> dict:
    """{(flags, n): (warps_per_block, chunks_per_warp)} for every even n in
    2..HAF_MAX_N, from the nearest tabulated size below (else the smallest)."""
    by_flags: dict = {}
    for e in table.get("entries", []):
        by_flags.setdefault(int(e["flags"]), []).append(e)
    out = {}
    for flags, es in by_flags.items():
        es = sorted(es, key=lambda e: e["n"])
        for n in range(2, _native.HAF_MAX_N + 1, 2):
            below = [e for e in es if e["n"] <= n]
            e = below[-1] if below else es[0]
            out[(flags, n)] = (int(e["warps_per_block"]), int(e["chunks_per_warp"]))
    return out


def load(path: str = TABLE_PATH) -> int:
    """Install a table into the library for haf and lhaf of every even n;
    returns the number of shapes installed (0 if there is no table)."""
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        table = json.load(f)
    L = _native.lib()
    k = 0
    for (flags, n), (wpb, cpw) in shapes(table).items():
        for loops in (0, _native.HAF_FLAG_LOOPS):
            _native.check(L.haf_tune_set(n, flags | loops, wpb, cpw))
            k += 1
    return k


def ensure_loaded() -> None:
    """Load the shipped table once (called before the first GPU call)."""
    global _loaded
    if not _loaded:
        _loaded = True
        load()


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE_PATH)
    ap.add_argument("--reps", type=int, default=1)
    a = ap.parse_args()
    generate(a.out, a.reps)
