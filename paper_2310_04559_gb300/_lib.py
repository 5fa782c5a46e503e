"""ctypes declarations for libcc_ladder.so (include/cc_ladder.h).

Argument marshalling only: every step of the ladder term runs in the CUDA
library.  Loading fails loudly when the library has not been built -- there is
no CPU or eager fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

CC_OK = 0
STATUS = {
    0: "CC_OK", -1: "CC_ERR_SHAPE", -2: "CC_ERR_NULL", -3: "CC_ERR_ALIGN", -4: "CC_ERR_WORKSPACE",
    -5: "CC_ERR_BUDGET", -6: "CC_ERR_UNSUPPORTED", -7: "CC_ERR_CUDA", -8: "CC_ERR_DEVICE_TIMEOUT", -9: "CC_ERR_ARG",
    -10: "CC_ERR_NOALLOC_LIMIT", -11: "CC_ERR_NONFINITE",
}
MODES = {"fp64": 0, "ozaki_bf16": 1, "ozaki_int8": 2, "tf32": 3, "bf16": 4}
ORDERS = {"auto": 0, "integral_first": 1, "cholesky_first": 2}
FLAG_ACCUMULATE, FLAG_SYMMETRIC_T, FLAG_EXCHANGE, FLAG_NO_STATUS_SYNC, FLAG_HOST_T2R, FLAG_HOST_L = 1, 2, 4, 8, 16, 32

_vp = ctypes.c_void_p
_sz = ctypes.c_size_t
_i = ctypes.c_int


class Args(ctypes.Structure):
    """struct cc_ladder_args"""
    _fields_ = [
        ("o", _i), ("v", _i), ("n_chol", _i),
        ("L", _vp), ("t2", _vp), ("R", _vp), ("energy", _vp),
        ("mode", _i), ("order", _i), ("a_block", _i), ("flags", _i), ("slices", _i),
        ("workspace", _vp), ("ws_bytes", _sz), ("budget_bytes", _sz), ("stream", _vp),
        ("a_lo", _i), ("a_hi", _i), ("chol_chunk", _i),
    ]


class Plan(ctypes.Structure):
    """struct cc_ladder_plan"""
    _fields_ = [
        ("order", _i), ("a_block", _i), ("n_blocks", _i), ("slices", _i), ("pairs", _i),
        ("ws_bytes", _sz), ("flops_algorithmic", ctypes.c_double), ("flops_issued", ctypes.c_double),
        ("pair_blocks", _i),
    ]


class ProfileEntry(ctypes.Structure):
    """struct cc_ladder_profile_entry"""
    _fields_ = [("name", ctypes.c_char * 32), ("launches", _i), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("bytes", ctypes.c_double)]


class LadderError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({strerror(status)})")


_lib = None

SYMBOLS = [
    "cc_ladder_workspace_size", "cc_ladder_workspace_size_ex", "cc_ladder_plan_query", "cc_ladder_fwd",
    "cc_ladder_fwd_ex", "cc_ladder_bwd_workspace_size", "cc_ladder_bwd", "cc_ladder_bwd_ex", "cc_ladder_energy",
    "cc_ladder_energy_workspace_size", "cc_ladder_device_status", "cc_ladder_set_wait_limit_ns",
    "cc_ladder_strerror", "cc_ladder_version", "cc_ladder_gemm_workspace_size", "cc_ladder_gemm",
    "cc_ladder_profile_enable", "cc_ladder_profile_read", "cc_ladder_launch_count", "cc_ladder_energy_noalloc",
    "cc_ladder_autotune", "cc_ladder_partition", "cc_ladder_peak_probe", "cc_ladder_term_workspace_size", "cc_ladder_term", "cc_ladder_tijkl", "cc_ladder_tijbk",
]
TERMS = {"ijkl": 1, "ijbk": 2}
PROBES = {"dmma": 1, "dfma": 2, "tc_bf16": 3, "tc_tf32": 4, "imma": 5}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libcc_ladder.so (building it first if allowed); raises if it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libcc_ladder.so not found at {path}; run paper_2310_04559_gb300.build.build()")
    L = ctypes.CDLL(path)
    L.cc_ladder_workspace_size.argtypes = [_i, _i, _i, _i, _sz, ctypes.POINTER(_sz)]
    L.cc_ladder_workspace_size_ex.argtypes = [ctypes.POINTER(Args), ctypes.POINTER(_sz)]
    L.cc_ladder_plan_query.argtypes = [ctypes.POINTER(Args), ctypes.POINTER(Plan)]
    L.cc_ladder_fwd.argtypes = [_i, _i, _i, _vp, _vp, _vp, _i, _vp, _vp, _sz, _vp]
    L.cc_ladder_fwd_ex.argtypes = [ctypes.POINTER(Args)]
    L.cc_ladder_bwd_workspace_size.argtypes = [_i, _i, _i, _i, _sz, ctypes.POINTER(_sz)]
    L.cc_ladder_bwd.argtypes = [_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, _sz, _vp]
    L.cc_ladder_bwd_ex.argtypes = [_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _vp, _sz, _vp]
    L.cc_ladder_energy.argtypes = [_i, _i, _vp, _vp, _vp, _vp, _vp, _sz, _vp]
    L.cc_ladder_energy_workspace_size.argtypes = [_i, _i, ctypes.POINTER(_sz)]
    L.cc_ladder_device_status.argtypes = [_vp, _vp]
    L.cc_ladder_set_wait_limit_ns.argtypes = [ctypes.c_ulonglong]
    L.cc_ladder_set_wait_limit_ns.restype = None
    L.cc_ladder_gemm_workspace_size.argtypes = [_i, _i, _i, _i, _i, ctypes.POINTER(_sz)]
    L.cc_ladder_gemm.argtypes = [_i, _i, _i, _i, _vp, _i, _vp, _i, _vp, _i, _i, _i, _vp, _sz, _vp]
    L.cc_ladder_profile_enable.argtypes = [_i]
    L.cc_ladder_profile_enable.restype = None
    L.cc_ladder_profile_read.argtypes = [ctypes.POINTER(ProfileEntry), _i]
    L.cc_ladder_launch_count.argtypes = []
    L.cc_ladder_launch_count.restype = ctypes.c_longlong
    L.cc_ladder_energy_noalloc.argtypes = [_i, _i, _vp, _vp, _vp, _vp, _vp]
    L.cc_ladder_autotune.argtypes = [ctypes.POINTER(Args), ctypes.POINTER(Plan), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
    L.cc_ladder_peak_probe.argtypes = [_i, _i, _vp, ctypes.POINTER(ctypes.c_double)]
    L.cc_ladder_partition.argtypes = [ctypes.POINTER(Args), _i, ctypes.POINTER(_i)]
    L.cc_ladder_term_workspace_size.argtypes = [_i, _i, _i, _i, _i, _i, _sz, ctypes.POINTER(_sz)]
    L.cc_ladder_term.argtypes = [_i, _i, _i, _i, _vp, _vp, _vp, _vp, _i, _i, _i, _vp, _sz, _vp]
    L.cc_ladder_tijkl.argtypes = [_i, _i, _i, _vp, _vp, _vp, _i, _vp, _sz, _vp]
    L.cc_ladder_tijbk.argtypes = [_i, _i, _i, _vp, _vp, _vp, _vp, _i, _vp, _sz, _vp]
    L.cc_ladder_strerror.argtypes = [_i]
    L.cc_ladder_strerror.restype = ctypes.c_char_p
    L.cc_ladder_version.restype = ctypes.c_char_p
    for name in SYMBOLS:
        if name not in ("cc_ladder_strerror", "cc_ladder_version", "cc_ladder_set_wait_limit_ns",
                        "cc_ladder_profile_enable", "cc_ladder_launch_count"):
            getattr(L, name).restype = _i
    _lib = L
    return L


def strerror(status: int) -> str:
    try:
        return load(build_if_missing=False).cc_ladder_strerror(status).decode()
    except Exception:  # noqa: BLE001 - message only
        return STATUS.get(status, "unknown")


def check(status: int, where: str):
    if status != CC_OK:
        raise LadderError(status, where)
