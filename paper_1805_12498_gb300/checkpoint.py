"""Checkpoint and resume for long hafnians.

The subset sum of Sec. 3.2 (eq. main) splits into independent parts: part p
of P takes a contiguous colex slice of every subset-size class
(``haf_part``).  Each part reduces to a 5-double record
{re_hi, im_hi, re_lo, im_lo, sum |f(Z)|}, and ``combine`` adds records in
part order in double-double.  A hafnian at n = 52-56 takes minutes, so
``run`` evaluates the parts one at a time. After each part it rewrites a
JSON record file: a temporary file in the same directory, then a rename.
A restarted ``run`` skips the parts the file already holds.

Failure detection:
- The file's header names the matrix (SHA-256 of its bytes in the dtype the
  library reads), loops, real, precision and P. A file whose header does not
  match raises ``ValueError`` instead of mixing two sums.
- Each record carries a SHA-256 of its 40 bytes. A record whose checksum
  fails, or that is not finite, is dropped and its part is evaluated again.
- Before the combine, the subset counts of the parts (``part_subsets``,
  host-only) must add up to 2^{n/2} - 1, so every subset is covered exactly
  once.

Every part runs on the GPU through ``haf_part``; this module only schedules
the parts and stores their records.
"""
from __future__ import annotations

import hashlib
import json
import os
import struct
import tempfile
from dataclasses import dataclass, field

import numpy as np

FORMAT = "haf-checkpoint-1"


@dataclass
class Progress:
    """State after a call of ``run``."""
    nparts: int
    done: list = field(default_factory=list)       # parts with a valid record, ascending
    computed: list = field(default_factory=list)   # parts evaluated by this call
    dropped: list = field(default_factory=list)    # records rejected on load (re-evaluated)
    value: complex | None = None                   # set once every part is done
    abs_sum: float | None = None

    @property
    def complete(self) -> bool:
        return len(self.done) == self.nparts


def _matrix_digest(A: np.ndarray) -> str:
    a = np.ascontiguousarray(A)
    h = hashlib.sha256()
    h.update(str(a.dtype.str).encode())
    h.update(struct.pack("<qq", *a.shape))
    h.update(a.astype(a.dtype.newbyteorder("<"), copy=False).tobytes())
    return h.hexdigest()


def _record_digest(rec) -> str:
    return hashlib.sha256(struct.pack("<5d", *[float(x) for x in rec])).hexdigest()


def _header(A: np.ndarray, loops: bool, real: bool, precision: str, nparts: int) -> dict:
    return {"format": FORMAT, "n": int(A.shape[0]), "loops": bool(loops), "real": bool(real),
            "precision": precision, "nparts": int(nparts), "matrix_sha256": _matrix_digest(A)}


def _load(path: str, header: dict):
    """Valid records {part: rec} and the list of dropped parts."""
    if not os.path.exists(path):
        return {}, []
    with open(path) as f:
        state = json.load(f)
    if state.get("header") != header:
        raise ValueError(f"checkpoint {path} belongs to another computation: {state.get('header')}")
    recs, dropped = {}, []
    for key, entry in state.get("records", {}).items():
        p = int(key)
        try:
            rec = [float.fromhex(x) for x in entry["rec"]]
            ok = (len(rec) == 5 and 0 <= p < header["nparts"] and entry.get("sha256") == _record_digest(rec)
                  and all(np.isfinite(rec)))
        except (KeyError, TypeError, ValueError):
            ok = False
        if ok:
            recs[p] = rec
        else:
            dropped.append(p)
    return recs, sorted(dropped)


def _save(path: str, header: dict, recs: dict) -> None:
    state = {"header": header,
             "records": {str(p): {"rec": [float(x).hex() for x in r], "sha256": _record_digest(r)}
                         for p, r in sorted(recs.items())}}
    d = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".haf-ckpt-", dir=d)
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(state, f, indent=1)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def run(A, path: str, nparts: int = 16, loops: bool = False, real: bool | None = None,
        precision: str = "fp64", parts=None) -> Progress:
    """Evaluate the parts of haf(A) (lhaf with ``loops``) not yet in the
    record file ``path``, saving after each one.  ``parts`` limits this call
    to the given part indices (default: every missing part).  Once every part
    has a record, the returned ``Progress`` carries the combined value and
    sum |f(Z)|."""
    import paper_1805_12498_gb300 as hg

    A = np.asarray(A)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square matrix")
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    if real is None:
        real = not np.iscomplexobj(A)
    A = np.ascontiguousarray(A, dtype=np.float64 if real else np.complex128)
    header = _header(A, loops, real, precision, nparts)
    recs, dropped = _load(path, header)
    todo = range(nparts) if parts is None else sorted(set(int(p) for p in parts))
    computed = []
    for p in todo:
        if not 0 <= p < nparts:
            raise ValueError(f"part {p} outside 0..{nparts - 1}")
        if p in recs:
            continue
        rec = np.asarray(hg.haf_part(A, p, nparts, loops=loops, real=real, precision=precision), dtype=np.float64)
        if rec.shape != (5,) or not np.all(np.isfinite(rec)):
            raise RuntimeError(f"part {p}: invalid record {rec!r}")
        recs[p] = [float(x) for x in rec]
        computed.append(p)
        _save(path, header, recs)
    prog = Progress(nparts=nparts, done=sorted(recs), computed=computed, dropped=dropped)
    if prog.complete:
        n = A.shape[0]
        n_eff = n + 1 if (n % 2 and loops) else n
        if n_eff % 2 == 0 and n_eff > 0:
            covered = sum(hg.part_subsets(n_eff, p, nparts) for p in range(nparts))
            if covered != 2 ** (n_eff // 2) - 1:
                raise RuntimeError(f"parts cover {covered} subsets, expected {2 ** (n_eff // 2) - 1}")
        prog.value, prog.abs_sum = hg.combine([recs[p] for p in range(nparts)])
    return prog
