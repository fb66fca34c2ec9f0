"""The oracle's pins catch plausible mistakes planted in the oracle.

Each case below copies the ``oracle`` package into a temporary directory,
plants ONE mistake in the copy (a dropped term, a wrong sign, index or
weight, a transposed operand), builds it, and runs the pin suite
``tests/test_oracle.py`` against it in a fresh interpreter.  The pins
must report a failed test (pytest exit code 1: an assertion, not a crash).
An unmodified copy, built and run the same way, must pass: that control
shows the failures come from the planted mistakes and not from the harness.

Everything here runs on the CPU; the repository's oracle is never modified.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")
PINS = os.path.join(ROOT, "tests", "test_oracle.py")

# (name, file, original snippet, planted snippet).  Each original snippet
# must occur exactly once in its file.
MUTANTS = [
    # --- Sec. 2: the definition by enumeration ---------------------------
    ("brute: loops never taken", "oracle.c",
     "if (ctx->loops) bf_rec(", "if (0) bf_rec("),
    ("brute: partner index starts one too late", "oracle.c",
     "for (int j = i + 1; j < ctx->n; j++) {", "for (int j = i + 2; j < ctx->n; j++) {"),
    ("brute: reads the lower triangle", "oracle.c",
     "int r = i < j ? i : j, c = i < j ? j : i;", "int r = i < j ? j : i, c = i < j ? i : j;"),
    ("complex product: wrong sign in the real part", "oracle.c",
     "a.re * b.re - a.im * b.im", "a.re * b.re + a.im * b.im"),
    # --- Sec. 3.3: B = (X A)^{(Z)} and the power traces -------------------
    ("B: pair swap X left out", "oracle.c",
     "int i = idx[r] ^ 1, j = idx[s];", "int i = idx[r], j = idx[s];"),
    ("B: diagonal of A kept as an edge", "oracle.c",
     "B[r * N + s] = (i == j) ? cq_mk(0, 0) : entry(A, n, i, j);",
     "B[r * N + s] = entry(A, n, i, j);"),
    ("traces: weight 1/k instead of 1/(2k)", "oracle.c",
     "c[k] = cq_scale(t, (quad)1 / (quad)(2 * k));", "c[k] = cq_scale(t, (quad)1 / (quad)k);"),
    ("powers: transposed left operand", "oracle.c",
     "cq_mul(P[r * N + l], B[l * N + s])", "cq_mul(P[l * N + r], B[l * N + s])"),
    # --- Sec. 3.3: the loop term q(lambda, B, v) ---------------------------
    ("loop term: weight 1 instead of 1/2", "oracle.c",
     "c[k] = cq_add(c[k], cq_scale(u, (quad)0.5));", "c[k] = cq_add(c[k], cq_scale(u, (quad)1.0));"),
    ("loop term: X left out of the start vector", "oracle.c",
     "for (int r = 0; r < N; r++) y[r] = v[r ^ 1];", "for (int r = 0; r < N; r++) y[r] = v[r];"),
    ("loop term: iterates with B transposed", "oracle.c",
     "cq b = (variant == 0) ? B[r * N + l] :", "cq b = (variant == 0) ? B[l * N + r] :"),
    # --- eq. poly: the truncated exponential ------------------------------
    ("exp series: 1/j! factor dropped", "oracle.c",
     "Q2[k] = cq_scale(acc, (quad)1 / (quad)j);", "Q2[k] = acc;"),
    ("exp series: linear term dropped", "oracle.c",
     "for (int k = 0; k <= h; k++) E[k] = Q[k];", "for (int k = 0; k <= h; k++) E[k] = cq_mk(0, 0);"),
    ("exp series: last power dropped", "oracle.c",
     "for (int j = 2; j <= h; j++) {", "for (int j = 2; j < h; j++) {"),
    ("exp series: coefficient index off by one", "oracle.c",
     "cq_mul(Q[a], c[k - a])", "cq_mul(Q[a], c[k - a + 1])"),
    # --- eq. main: the signed subset sum ----------------------------------
    ("subset sum: sign flipped", "oracle.c",
     "if ((h - m) & 1)", "if ((h - m + 1) & 1)"),
    ("subset sum: |Z| of the wrong mask", "oracle.c",
     "int m = __builtin_popcountll((unsigned long long)z);",
     "int m = __builtin_popcountll((unsigned long long)(z >> 1));"),
    ("subset sum: |f| from the real part only", "oracle.c",
     "t_abs += hypot((double)f.re, (double)f.im);", "t_abs += fabs((double)f.re);"),
    # --- Ryser (eq. bipartite) --------------------------------------------
    ("Ryser: sign from |S| instead of k - |S|", "oracle.c",
     "if ((k - sz) & 1)", "if (sz & 1)"),
    ("Ryser: imaginary parts dropped", "oracle.c",
     "(quad)W[2 * (i * k + j) + 1]", "(quad)0"),
    # --- App. A and App. C (Python side of the oracle) --------------------
    ("telephone: recurrence weight k instead of k - 1", "__init__.py",
     "t.append(t[k - 1] + (k - 1) * t[k - 2])", "t.append(t[k - 1] + k * t[k - 2])"),
    ("double factorial: steps of one", "__init__.py",
     "        a -= 2\n", "        a -= 1\n"),
    ("low rank: (e - 1)!! replaced by e!!", "__init__.py",
     "w *= double_factorial(x - 1)", "w *= double_factorial(x)"),
    ("low rank: odd exponent vectors kept", "__init__.py",
     "if all(x % 2 == 0 for x in e):", "if True:"),
]

_RUNNER = (
    "import sys\n"
    "sys.path.insert(0, sys.argv[1])\n"
    "import oracle\n"
    "assert oracle.__file__.startswith(sys.argv[1]), oracle.__file__\n"
    "oracle.build.build(force=True)\n"
    "import pytest\n"
    "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', sys.argv[2]]))\n"
)


def _copy_with(tmp, fname=None, old=None, new=None):
    """Copy the oracle package's sources into tmp/oracle, with one snippet
    replaced in one file; return the directory to put on sys.path."""
    dst = os.path.join(tmp, "oracle")
    os.makedirs(dst)
    for f in ("__init__.py", "build.py", "oracle.c"):
        shutil.copy(os.path.join(ORACLE_DIR, f), os.path.join(dst, f))
    if fname is not None:
        path = os.path.join(dst, fname)
        with open(path) as fh:
            src = fh.read()
        assert src.count(old) == 1, f"snippet not unique in {fname}: {old!r}"
        with open(path, "w") as fh:
            fh.write(src.replace(old, new))
    return tmp


def _run_pins(pkg_parent):
    return subprocess.run([sys.executable, "-c", _RUNNER, pkg_parent, PINS], cwd=ROOT,
                          capture_output=True, text=True, timeout=300)


def test_snippets_are_unique_in_the_oracle():
    for name, fname, old, _ in MUTANTS:
        with open(os.path.join(ORACLE_DIR, fname)) as fh:
            assert fh.read().count(old) == 1, name


def test_unmodified_copy_passes_the_pins(tmp_path):
    r = _run_pins(_copy_with(str(tmp_path)))
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    def one(i):
        name, fname, old, new = MUTANTS[i]
        d = os.path.join(str(tmp_path), f"m{i}")
        os.makedirs(d)
        r = _run_pins(_copy_with(d, fname, old, new))
        return name, r

    with ThreadPoolExecutor(max_workers=min(4, os.cpu_count() or 1)) as ex:
        results = list(ex.map(one, range(len(MUTANTS))))
    survivors = [name for name, r in results if r.returncode == 0]
    assert not survivors, f"planted mistakes no pin caught: {survivors}"
    crashed = [(name, r.returncode, r.stderr[-500:]) for name, r in results if r.returncode != 1]
    assert not crashed, f"mutants that did not end in a failed pin: {crashed}"
