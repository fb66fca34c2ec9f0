"""ctypes binding of the C ABI in include/hafnian_gb300.h (argument
marshalling only: every step of the hafnian runs in the CUDA library).

The shared library is built in-tree by ``paper_1805_12498_gb300.build``;
if it is missing and cannot be built, every call raises instead of falling
back to any CPU path.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

HAF_OK = 0
HAF_EINVAL = -1
HAF_ENOMEM = -2
HAF_ECUDA = -3
HAF_ETIMEDOUT = -4
HAF_EBUSY = -5
HAF_ENOTFOUND = -6
HAF_ESMALL = -7
HAF_EACCURACY = -8
HAF_FLAG_LOOPS = 1
HAF_FLAG_REAL = 2
HAF_FLAG_FP32 = 4
HAF_MAX_N = 56


class HafInfo(ctypes.Structure):
    _fields_ = [("abs_sum", ctypes.c_double), ("value_lo", ctypes.c_double * 2),
                ("subsets", ctypes.c_int64), ("seconds", ctypes.c_double),
                ("launches", ctypes.c_int64), ("rel_err_bound", ctypes.c_double),
                ("precision_mode", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int32), ("chunks_per_warp", ctypes.c_int32),
                ("ms", ctypes.c_double), ("ms_default", ctypes.c_double), ("candidates", ctypes.c_int32)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("max_jobs", ctypes.c_int64), ("max_bytes", ctypes.c_int64),
                ("ring_entries", ctypes.c_int64), ("idle_us", ctypes.c_int64), ("chunk_us", ctypes.c_int64)]


class HafError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hafnian_gb300 error {code}: {msg}")
        self.code = code


class HafAccuracyError(HafError):
    """An FP32-bulk result whose estimated relative error exceeds
    HAF_FP32_MAX_REL_ERR (HAF_EACCURACY).  ``result`` holds the value and
    report the library wrote anyway (set by the caller that raises it)."""
    result = None


_lib = None
_lock = threading.Lock()

_DP = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)
_U64P = ctypes.POINTER(ctypes.c_uint64)


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run paper_1805_12498_gb300.build")
        L = ctypes.CDLL(path)
        for name in ("haf_c128", "lhaf_c128", "haf_f64", "lhaf_f64"):
            f = getattr(L, name)
            f.argtypes = [_DP, ctypes.c_int64, _DP, ctypes.POINTER(HafInfo)]
            f.restype = ctypes.c_int
        for name in ("haf_c128_batched", "lhaf_c128_batched"):
            f = getattr(L, name)
            f.argtypes = [ctypes.POINTER(_DP), _I64P, ctypes.c_int64, _DP, ctypes.POINTER(HafInfo)]
            f.restype = ctypes.c_int
        L.haf_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_uint32]
        L.haf_workspace_bytes.restype = ctypes.c_size_t
        L.haf_launch.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p,
                                 ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
        L.haf_launch.restype = ctypes.c_int
        L.haf_launch_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p,
                                         ctypes.c_void_p]
        L.haf_launch_noalloc.restype = ctypes.c_int
        L.haf_terms_c128.argtypes = [_DP, ctypes.c_int64, ctypes.c_int, _U64P, ctypes.c_int64, _DP]
        L.haf_terms_c128.restype = ctypes.c_int
        L.haf_terms.argtypes = [_DP, ctypes.c_int64, ctypes.c_uint32, _U64P, ctypes.c_int64, _DP]
        L.haf_terms.restype = ctypes.c_int
        L.haf_lowrank_c128.argtypes = [_DP, ctypes.c_int64, ctypes.c_int64, _DP, ctypes.POINTER(HafInfo)]
        L.haf_lowrank_c128.restype = ctypes.c_int
        L.haf_lowrank_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int64]
        L.haf_lowrank_workspace_bytes.restype = ctypes.c_size_t
        L.haf_lowrank_launch.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
        L.haf_lowrank_launch.restype = ctypes.c_int
        L.haf_eval.argtypes = [_DP, ctypes.c_int64, ctypes.c_uint32, _DP, ctypes.POINTER(HafInfo)]
        L.haf_eval.restype = ctypes.c_int
        L.haf_batched.argtypes = [ctypes.POINTER(_DP), _I64P, ctypes.c_int64, ctypes.c_uint32, _DP,
                                  ctypes.POINTER(HafInfo)]
        L.haf_batched.restype = ctypes.c_int
        L.haf_tune.argtypes = [ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32, ctypes.POINTER(TuneResult)]
        L.haf_tune.restype = ctypes.c_int
        L.haf_plan_stats.argtypes = [ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32, _I64P]
        L.haf_plan_stats.restype = ctypes.c_int
        L.haf_tune_set.argtypes = [ctypes.c_int64, ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32]
        L.haf_tune_set.restype = ctypes.c_int
        L.haf_batched_tune.argtypes = [ctypes.POINTER(_DP), _I64P, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_int32, ctypes.POINTER(TuneResult)]
        L.haf_batched_tune.restype = ctypes.c_int
        L.haf_part.argtypes = [_DP, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64, _DP,
                               ctypes.POINTER(HafInfo)]
        L.haf_part.restype = ctypes.c_int
        L.haf_part_subsets.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _I64P]
        L.haf_part_subsets.restype = ctypes.c_int
        L.haf_combine.argtypes = [_DP, ctypes.c_int64, _DP]
        L.haf_combine.restype = ctypes.c_int
        L.haf_server_create.argtypes = [ctypes.POINTER(ServerCfg), ctypes.POINTER(ctypes.c_void_p)]
        L.haf_server_create.restype = ctypes.c_int
        L.haf_server_submit.argtypes = [ctypes.c_void_p, ctypes.c_int, _DP, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_uint64)]
        L.haf_server_submit.restype = ctypes.c_int
        L.haf_server_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, _DP, ctypes.POINTER(HafInfo),
                                      ctypes.c_int64]
        L.haf_server_poll.restype = ctypes.c_int
        L.haf_server_destroy.argtypes = [ctypes.c_void_p]
        L.haf_server_destroy.restype = ctypes.c_int
        L.haf_fp64_peak.argtypes = [_DP, _DP]
        L.haf_fp64_peak.restype = ctypes.c_int
        L.haf_last_error.argtypes = []
        L.haf_last_error.restype = ctypes.c_char_p
        L.haf_version.argtypes = []
        L.haf_version.restype = ctypes.c_char_p
        _lib = L
        return L


def check(rc: int) -> None:
    if rc != HAF_OK:
        msg = lib().haf_last_error()
        cls = HafAccuracyError if rc == HAF_EACCURACY else HafError
        raise cls(rc, msg.decode() if msg else "")
