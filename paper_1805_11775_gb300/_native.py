"""ctypes binding of ``libhos.so`` (the C ABI declared in include/hos.h).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels.  Loading fails loudly if the library is not built.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
# HOS_LIB selects another build of the library (the bounds-checking variant,
# _lib/libhos_debug_bounds.so); the default is the in-tree libhos.so
LIB_PATH = os.environ.get("HOS_LIB") or os.path.join(_PKG, "_lib", "libhos.so")

HOS_OK = 0
STATUS_NAMES = {0: "HOS_OK", 1: "HOS_ERR_INVALID_ARG", 2: "HOS_ERR_UNSUPPORTED", 3: "HOS_ERR_WORKSPACE",
                4: "HOS_ERR_CUDA", 5: "HOS_ERR_TIMEOUT", 6: "HOS_ERR_DEVICE_FAULT"}
F32, F64 = 0, 1
(OP_BISPECTRUM, OP_TRISPECTRUM, OP_BISPECTRUM_BATCHED, OP_BISPECTRUM_BACKWARD, OP_CUMULANT3, OP_CUMULANT4,
 OP_SERIES_SUM, OP_CUMULANT3_SLICE, OP_BISPECTRUM_FROM_C3, OP_TRISPECTRUM_BATCHED, OP_TRISPECTRUM_BACKWARD,
 OP_MOMENTS4_SLICE, OP_TRISPECTRUM_FROM_MOMENTS) = range(13)


class HosParams(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("nfft", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("window", ctypes.c_int32), ("remove_mean", ctypes.c_int32), ("segment_len", ctypes.c_int32),
                ("tile_n", ctypes.c_int32), ("flush_chunks", ctypes.c_int32), ("segment_overlap", ctypes.c_int32),
                ("chunk_len", ctypes.c_int32)]


class HosError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} ({_string(status)})")


_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_P = ctypes.POINTER(HosParams)
_SIGS = {
    "hos_workspace_size": [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, _P,
                           ctypes.POINTER(ctypes.c_size_t)],
    "hos_bispectrum": [_VP, ctypes.c_int32, ctypes.c_int64, _P, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_trispectrum": [_VP, ctypes.c_int32, ctypes.c_int64, _P, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_bispectrum_batched": [_VP, ctypes.c_int32, _VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P, _VP,
                               _VP, ctypes.c_size_t, _VP],
    "hos_bispectrum_backward": [_VP, ctypes.c_int32, ctypes.c_int64, _P, _VP, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_trispectrum_backward": [_VP, ctypes.c_int32, ctypes.c_int64, _P, _VP, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_moments4_slice": [_VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_int64, _P,
                           _VP, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_trispectrum_from_moments": [_VP, _VP, _P, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_bispectrum_noalloc": [_VP, ctypes.c_int32, ctypes.c_int64, _P, _VP, _VP],
    "hos_bispectrum_noalloc_status": [ctypes.POINTER(ctypes.c_int32)],
    "hos_cumulant3": [_VP, ctypes.c_int32, ctypes.c_int64, _P, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_cumulant4": [_VP, ctypes.c_int32, ctypes.c_int64, _P, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_trispectrum_batched": [_VP, ctypes.c_int32, _VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, _P, _VP,
                                _VP, ctypes.c_size_t, _VP],
    "hos_series_sum": [_VP, ctypes.c_int32, ctypes.c_int64, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_cumulant3_slice": [_VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_int64,
                            _P, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_bispectrum_from_cumulant": [_VP, _P, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_bispectrum_direct_workspace_size": [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_size_t)],
    "hos_bispectrum_direct": [_VP, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                              ctypes.c_int32, _VP, _VP, ctypes.c_size_t, _VP],
    "hos_check_plan": [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, _VP, _P, ctypes.c_int32, ctypes.c_char_p,
                       ctypes.c_size_t],
    "hos_get_device_status": [_VP, ctypes.POINTER(ctypes.c_int32)],
    "hos_reset_device_status": [_VP, _VP],
    "hos_selftest_timeout": [_VP, ctypes.c_size_t, ctypes.c_int32, _VP],
    "hos_set_profiling": [ctypes.c_int32],
    "hos_get_stage_times": [ctypes.POINTER(ctypes.c_float), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)],
    "hos_stage_name": [ctypes.c_int32],
    "hos_launch_count": [],
    "hos_last_contraction": [],
    "hos_last_plan": [],
    "hos_status_string": [ctypes.c_int32],
    "hos_version": [],
}
_RESTYPES = {"hos_stage_name": ctypes.c_char_p, "hos_last_contraction": ctypes.c_char_p,
             "hos_last_plan": ctypes.c_char_p,
             "hos_status_string": ctypes.c_char_p, "hos_version": ctypes.c_char_p,
             "hos_launch_count": ctypes.c_int64}


def lib():
    """The loaded library; raises if libhos.so has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with "
                                  "`python -m paper_1805_11775_gb300.build` (needs nvcc)")
            h = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(h, name)
                fn.argtypes = args
                fn.restype = _RESTYPES.get(name, ctypes.c_int32)
            _lib = h
    return _lib


def _string(status: int) -> str:
    try:
        return lib().hos_status_string(int(status)).decode()
    except Exception:  # pragma: no cover
        return "?"


def check(status: int, where: str) -> None:
    if status != HOS_OK:
        raise HosError(status, where)
