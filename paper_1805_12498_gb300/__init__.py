"""GB300-native (sm_103a) hafnian and loop hafnian.

Python front end of the C ABI in include/hafnian_gb300.h.  Every number is
computed by the CUDA library; this module only marshals arguments.

    >>> import numpy as np, paper_1805_12498_gb300 as hg
    >>> hg.haf(np.ones((16, 16)))            # (16-1)!! = 2027025
    >>> hg.lhaf(np.ones((16, 16)))           # T(16) = 46206736

The hafnian is the sum over perfect matchings of the products of the
matched entries (Sec. 2); it is evaluated with the O(n^3 2^{n/2}) signed
subset sum of Sec. 3 on the GPU in FP64 with double-double accumulation.
``precision="fp32"`` selects the FP32-bulk mode (single-precision
reduction and La Budde recurrence, FP64 series and sum; n <= HAF_FP32_MAX_N).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _native, tuning
from ._native import (HAF_FLAG_FP32, HAF_FLAG_LOOPS, HAF_FLAG_REAL, HAF_MAX_N, HafAccuracyError,  # noqa: F401
                      HafError)

__all__ = ["haf", "lhaf", "haf_info", "haf_batched", "haf_terms", "workspace_bytes",
           "haf_launch", "haf_launch_noalloc", "haf_part", "part_subsets", "combine", "Server", "fp64_peak", "tune",
           "tune_set", "batched_tune", "haf_lowrank", "haf_lowrank_launch", "lowrank_workspace_bytes", "HafError", "HafAccuracyError", "HAF_MAX_N",
           "HAF_FP32_MAX_N", "HAF_FP32_REL_TOL", "HAF_FP64_REL_TOL", "HAF_FP32_MAX_REL_ERR"]

# Accuracy constants of include/hafnian_gb300.h: the error per unit of
# abs_sum measured against the oracle (FP64, FP32-bulk) and the bound on the
# estimated relative error above which an FP32-bulk result is refused.
HAF_FP32_MAX_N = 56
HAF_FP64_REL_TOL = 1e-13
HAF_FP32_REL_TOL = 3e-5
HAF_FP32_MAX_REL_ERR = 1e-3


def _flags(loops: bool = False, real: bool = False, precision: str = "fp64") -> int:
    if precision not in ("fp64", "fp32"):
        raise ValueError("precision must be 'fp64' or 'fp32'")
    return ((HAF_FLAG_LOOPS if loops else 0) | (HAF_FLAG_REAL if real else 0)
            | (HAF_FLAG_FP32 if precision == "fp32" else 0))


@dataclass
class Info:
    value: complex
    abs_sum: float
    value_lo: complex
    subsets: int
    seconds: float
    launches: int
    rel_err_bound: float = 0.0  # estimated |error| / |value| (0: not computed)
    precision_mode: int = 0     # 0: FP64, 1: FP32-bulk


def _info(value, info) -> Info:
    return Info(value, info.abs_sum, complex(info.value_lo[0], info.value_lo[1]), info.subsets, info.seconds,
                info.launches, info.rel_err_bound, info.precision_mode)


def _prep(A, real: bool) -> np.ndarray:
    A = np.asarray(A)
    if A.ndim != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square matrix")
    return np.ascontiguousarray(A, dtype=np.float64 if real else np.complex128)


def haf_info(A, loops: bool = False, real: bool | None = None, precision: str = "fp64") -> Info:
    """Hafnian (or loop hafnian) of A with the per-call report."""
    tuning.ensure_loaded()
    if real is None:
        real = not np.iscomplexobj(A)
    A = _prep(A, real)
    L = _native.lib()
    out = np.zeros(2)
    info = _native.HafInfo()
    if precision == "fp64":
        fn = {(False, False): L.haf_c128, (True, False): L.lhaf_c128,
              (False, True): L.haf_f64, (True, True): L.lhaf_f64}[(bool(loops), bool(real))]
        rc = fn(A.ctypes.data_as(_native._DP), A.shape[0], out.ctypes.data_as(_native._DP), ctypes.byref(info))
    else:
        rc = L.haf_eval(A.ctypes.data_as(_native._DP), A.shape[0], _flags(loops, real, precision),
                        out.ctypes.data_as(_native._DP), ctypes.byref(info))
    result = _info(complex(out[0], 0.0 if real else out[1]), info)
    try:
        _native.check(rc)
    except HafAccuracyError as e:
        e.result = result  # the refused FP32-bulk value and its report
        raise
    return result


def haf(A, loops: bool = False, precision: str = "fp64"):
    """haf(A) (Sec. 2, eq. hafA).  Real input gives a float, complex a complex."""
    r = haf_info(A, loops, precision=precision)
    return r.value.real if not np.iscomplexobj(A) else r.value


def lhaf(A, precision: str = "fp64"):
    """Loop hafnian lhaf(A) (Sec. 2)."""
    return haf(A, loops=True, precision=precision)


def _batch_args(mats):
    mats = [_prep(M, False) for M in mats]
    count = len(mats)
    ptrs = (_native._DP * max(1, count))(*[M.ctypes.data_as(_native._DP) for M in mats])
    ns = np.array([M.shape[0] for M in mats], dtype=np.int64)
    return mats, count, ptrs, ns


def haf_batched(mats, loops: bool = False, with_info: bool = False, precision: str = "fp64"):
    """Hafnians of a list of complex matrices of mixed sizes in one launch."""
    tuning.ensure_loaded()
    mats, count, ptrs, ns = _batch_args(mats)
    outs = np.zeros(2 * max(1, count))
    infos = (_native.HafInfo * max(1, count))()
    L = _native.lib()
    rc = L.haf_batched(ptrs, ns.ctypes.data_as(_native._I64P), count, _flags(loops, False, precision),
                       outs.ctypes.data_as(_native._DP), infos)
    vals = outs[0:2 * count:2] + 1j * outs[1:2 * count:2]
    result = [_info(complex(vals[i]), infos[i]) for i in range(count)]
    try:
        _native.check(rc)
    except HafAccuracyError as e:
        e.result = (vals, result)
        raise
    if not with_info:
        return vals
    return vals, result


def haf_terms(A, masks, loops: bool = False, precision: str = "fp64") -> np.ndarray:
    """Unsigned summands f(Z) for the given subset bitmasks (Sec. 3.3),
    computed with the launch shape a whole-matrix call of this size uses."""
    tuning.ensure_loaded()
    A = _prep(A, False)
    masks = np.ascontiguousarray(np.asarray(masks, dtype=np.uint64))
    out = np.zeros(2 * max(1, masks.size))
    _native.check(_native.lib().haf_terms(
        A.ctypes.data_as(_native._DP), A.shape[0], _flags(loops, False, precision),
        masks.ctypes.data_as(_native._U64P), masks.size, out.ctypes.data_as(_native._DP)))
    return out[0:2 * masks.size:2] + 1j * out[1:2 * masks.size:2]


def workspace_bytes(n: int, loops: bool = False, real: bool = False, precision: str = "fp64") -> int:
    tuning.ensure_loaded()
    flags = _flags(loops, real, precision)
    b = _native.lib().haf_workspace_bytes(n, flags)
    if b == 0:
        raise HafError(_native.HAF_EINVAL, f"no workspace size for n={n}")
    return int(b)


def haf_launch(dA_ptr: int, n: int, d_out_ptr: int, d_work_ptr: int, ws_bytes: int,
               stream_ptr: int = 0, loops: bool = False, real: bool = False, precision: str = "fp64") -> None:
    """Enqueue a hafnian on device memory (raw pointers, e.g. torch
    ``tensor.data_ptr()`` and ``torch.cuda.current_stream().cuda_stream``).
    The 5-double record {re_hi, im_hi, re_lo, im_lo, abs_sum} lands at
    d_out_ptr when the stream reaches it."""
    tuning.ensure_loaded()
    flags = _flags(loops, real, precision)
    _native.check(_native.lib().haf_launch(dA_ptr, n, flags, d_out_ptr, d_work_ptr, ws_bytes, stream_ptr))


def haf_launch_noalloc(dA_ptr: int, n: int, d_out_ptr: int, stream_ptr: int = 0, loops: bool = False,
                       real: bool = False) -> None:
    """Allocation-free form of ``haf_launch`` (FP64), for callers that may
    not allocate device memory at call time: the library's one static device
    scratch array takes the place of the workspace, and no call allocates.
    Calls that overlap on the GPU share that array and race, so keep them on
    one stream.  The same 5-double record lands at d_out_ptr."""
    flags = _flags(loops, real)
    _native.check(_native.lib().haf_launch_noalloc(dA_ptr, n, flags, d_out_ptr, stream_ptr))


def haf_part(A, part: int, nparts: int, loops: bool = False, real: bool | None = None,
             precision: str = "fp64", with_info: bool = False):
    """Record {re_hi, im_hi, re_lo, im_lo, abs_sum} of part `part` of `nparts`
    of the subset sum (each size class cut into nparts contiguous slices);
    runs on the current CUDA device.  Combine the parts with ``combine``.
    With ``with_info`` also the call's report (subsets, seconds, launches)."""
    tuning.ensure_loaded()
    if real is None:
        real = not np.iscomplexobj(A)
    A = _prep(A, real)
    flags = _flags(loops, real, precision)
    rec = np.zeros(5)
    info = _native.HafInfo()
    _native.check(_native.lib().haf_part(A.ctypes.data_as(_native._DP), A.shape[0], flags, part, nparts,
                                         rec.ctypes.data_as(_native._DP), ctypes.byref(info)))
    if with_info:
        return rec, _info(complex(rec[0] + rec[2], rec[1] + rec[3]), info)
    return rec


def part_subsets(n: int, part: int, nparts: int) -> int:
    """Number of subset terms that part `part` of `nparts` evaluates (host only)."""
    out = ctypes.c_int64()
    _native.check(_native.lib().haf_part_subsets(n, part, nparts, ctypes.byref(out)))
    return out.value


def combine(records) -> tuple[complex, float]:
    """Fixed-order double-double sum of part records (host only):
    returns (value, abs_sum)."""
    recs = np.ascontiguousarray(np.asarray(records, dtype=np.float64).reshape(-1, 5))
    out = np.zeros(5)
    _native.check(_native.lib().haf_combine(recs.ctypes.data_as(_native._DP), recs.shape[0],
                                            out.ctypes.data_as(_native._DP)))
    return complex(out[0] + out[2], out[1] + out[3]), float(out[4])


class Server:
    """Continuous-batching hafnian server on the current GPU (C ABI
    haf_server_*): submit haf/lhaf requests of mixed n while others run,
    collect each result once with ``poll``."""

    def __init__(self, max_jobs: int = 0, max_bytes: int = 0, ring_entries: int = 0, idle_us: int = 0,
                 chunk_us: int = 0):
        self._L = _native.lib()
        cfg = _native.ServerCfg(max_jobs, max_bytes, ring_entries, idle_us, chunk_us)
        h = ctypes.c_void_p()
        _native.check(self._L.haf_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, A, loops: bool = False) -> int:
        A = _prep(A, False)
        t = ctypes.c_uint64()
        _native.check(self._L.haf_server_submit(self._h, 1 if loops else 0, A.ctypes.data_as(_native._DP),
                                                A.shape[0], ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_s: float | None = None) -> Info:
        out = np.zeros(2)
        info = _native.HafInfo()
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        _native.check(self._L.haf_server_poll(self._h, ticket, out.ctypes.data_as(_native._DP),
                                               ctypes.byref(info), us))
        return _info(complex(out[0], out[1]), info)

    def close(self) -> None:
        if self._h:
            _native.check(self._L.haf_server_destroy(self._h))
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def haf_lowrank(G) -> Info:
    """haf(G G^T) for an n x r matrix G by the App. C expansion (rank-r
    inputs; polynomial in n for fixed r).  Only G G^T above the diagonal
    matters, so any G with G G^T = A + (lower triangular) gives haf(A)."""
    G = np.asarray(G)
    if G.ndim != 2:
        raise ValueError("G must be an n x r matrix")
    G = np.ascontiguousarray(G, dtype=np.complex128)
    out = np.zeros(2)
    info = _native.HafInfo()
    _native.check(_native.lib().haf_lowrank_c128(G.ctypes.data_as(_native._DP), G.shape[0], G.shape[1],
                                                 out.ctypes.data_as(_native._DP), ctypes.byref(info)))
    return _info(complex(out[0], out[1]), info)


def lowrank_workspace_bytes(n: int, r: int) -> int:
    """Device workspace of ``haf_lowrank_launch`` for an n x r matrix G."""
    b = _native.lib().haf_lowrank_workspace_bytes(n, r)
    if b == 0:
        raise HafError(_native.HAF_EINVAL, f"no low-rank workspace size for n={n}, r={r}")
    return int(b)


def haf_lowrank_launch(dG_ptr: int, n: int, r: int, d_out_ptr: int, d_work_ptr: int, ws_bytes: int,
                       stream_ptr: int = 0) -> None:
    """Enqueue the App. C expansion for G (complex128, row-major n x r) in
    device memory; the 5-double record {re_hi, im_hi, re_lo, im_lo,
    abs_sum} lands at d_out_ptr when the stream reaches it."""
    _native.check(_native.lib().haf_lowrank_launch(dG_ptr, n, r, d_out_ptr, d_work_ptr, ws_bytes, stream_ptr))


def tune(n: int, loops: bool = False, real: bool = False, precision: str = "fp64", reps: int = 1) -> dict:
    """Time every launch shape for a hafnian of size n with these flags and
    keep the fastest for later calls (haf_tune).  Returns the chosen shape
    and the times of it and of the default shape."""
    r = _native.TuneResult()
    _native.check(_native.lib().haf_tune(n, _flags(loops, real, precision), reps, ctypes.byref(r)))
    return {"warps_per_block": r.warps_per_block, "chunks_per_warp": r.chunks_per_warp, "ms": r.ms,
            "ms_default": r.ms_default, "candidates": r.candidates}


def tune_set(n: int, warps_per_block: int, chunks_per_warp: int, loops: bool = False, real: bool = False,
             precision: str = "fp64") -> None:
    """Record a launch shape for (n, flags) without timing (haf_tune_set)."""
    _native.check(_native.lib().haf_tune_set(n, _flags(loops, real, precision), warps_per_block,
                                             chunks_per_warp))


def batched_tune(mats, loops: bool = False, precision: str = "fp64", reps: int = 1) -> dict:
    """Tune the launch shape of one batch (its size list and flags) by timing
    graph replays of the whole batch (haf_batched_tune)."""
    mats, count, ptrs, ns = _batch_args(mats)
    r = _native.TuneResult()
    _native.check(_native.lib().haf_batched_tune(ptrs, ns.ctypes.data_as(_native._I64P), count,
                                                 _flags(loops, False, precision), reps, ctypes.byref(r)))
    return {"warps_per_block": r.warps_per_block, "chunks_per_warp": r.chunks_per_warp, "ms": r.ms,
            "ms_default": r.ms_default, "candidates": r.candidates}


def fp64_peak() -> tuple[float, float]:
    """(TFLOP/s, ms) of the library's DFMA throughput probe on this GPU."""
    t = ctypes.c_double()
    ms = ctypes.c_double()
    _native.check(_native.lib().haf_fp64_peak(ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def version() -> str:
    return _native.lib().haf_version().decode()
