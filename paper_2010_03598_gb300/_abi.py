"""ctypes declarations mirroring include/kgrape.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkgrape.so")

KG_OK, KG_ERR_INVALID_ARG, KG_ERR_UNSUPPORTED, KG_ERR_CUDA, KG_ERR_NONFINITE, KG_ERR_TIMEOUT, KG_ERR_WORKSPACE = range(7)
STATUS_NAMES = {0: "KG_OK", 1: "KG_ERR_INVALID_ARG", 2: "KG_ERR_UNSUPPORTED", 3: "KG_ERR_CUDA",
                4: "KG_ERR_NONFINITE", 5: "KG_ERR_TIMEOUT", 6: "KG_ERR_WORKSPACE"}
KG_PREC_C128, KG_PREC_C64_F64REC, KG_PREC_FF = 0, 1, 2
KG_GRAD_NONE, KG_GRAD_CENTERED, KG_GRAD_ZEROTH, KG_GRAD_EXACT, KG_GRAD_TAYLOR1, KG_GRAD_TAYLOR2 = 0, 1, 2, 3, 4, 5
KG_HC_SX_SITE, KG_HC_SZ_SITES = 0, 1
KG_FLAG_HOST_STAGING = 1
KG_FLAG_PHASE_TIMING = 2
KG_FLAG_FULL_REORTH = 4
KG_CKPT_AUTO = -1
KG_STATIC_WORKSPACE_BYTES = 64 << 20


class KgChain(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("hc_kind", ctypes.c_int32), ("hc_site", ctypes.c_int32),
                ("reserved0", ctypes.c_int32), ("hc_site_mask", ctypes.c_uint64), ("Jxy", ctypes.c_double),
                ("Jz", ctypes.c_double), ("hc_amp", ctypes.c_double)]


class KgOptions(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("m", ctypes.c_int32), ("prec", ctypes.c_int32), ("grad", ctypes.c_int32),
                ("ckpt_every", ctypes.c_int32), ("tile_bits", ctypes.c_int32), ("ctas", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("dt", ctypes.c_double), ("breakdown_tol", ctypes.c_double),
                ("mem_budget", ctypes.c_int64)]


class KgReport(ctypes.Structure):
    _fields_ = [("krylov_err_max", ctypes.c_double), ("norm_final", ctypes.c_double), ("beta_re", ctypes.c_double),
                ("beta_im", ctypes.c_double), ("breakdowns", ctypes.c_int32), ("status", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("ctas", ctypes.c_int32), ("tile_bits", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("ckpt_every", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("phase_cycles", ctypes.c_int64 * 8)]


class KgBatchSchedule(ctypes.Structure):
    _fields_ = [("ctas", ctypes.c_int32), ("tiles_per_cta", ctypes.c_int32), ("reserved0", ctypes.c_int32),
                ("reserved1", ctypes.c_int32)]


class KgSector(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("K", ctypes.c_int32), ("parity", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("hc_site_mask", ctypes.c_uint64), ("Jxy", ctypes.c_double),
                ("Jz", ctypes.c_double), ("hc_amp", ctypes.c_double)]


_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); one entry per function declared in include/kgrape.h
SIGNATURES = {
    "kg_version": (ctypes.c_int, []),
    "kg_last_error": (ctypes.c_char_p, []),
    "kg_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(KgChain), ctypes.POINTER(KgOptions),
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "kg_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(KgChain), ctypes.POINTER(KgOptions), _P,
                                 ctypes.c_size_t, _P]),
    "kg_evaluate": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "kg_evaluate_host": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "kg_sync": (ctypes.c_int, [_P, ctypes.POINTER(KgReport)]),
    "kg_destroy": (ctypes.c_int, [_P]),
    "kg_set_wait_limit_ns": (ctypes.c_int, [ctypes.c_int64]),
    "kg_debug_set_fault": (ctypes.c_int, [ctypes.c_int32]),
    "kg_batch_workspace_bytes": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(KgChain), ctypes.POINTER(KgOptions),
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "kg_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.POINTER(KgChain),
                                       ctypes.POINTER(KgOptions), ctypes.POINTER(KgBatchSchedule), _P, _P, _P, _P, _P,
                                       _P, ctypes.c_size_t, _P]),
    "kg_batch_launch": (ctypes.c_int, [_P]),
    "kg_batch_sync": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "kg_batch_destroy": (ctypes.c_int, [_P]),
    "kg_evaluate_static": (ctypes.c_int, [ctypes.POINTER(KgChain), ctypes.POINTER(KgOptions), _P, _P, _P, _P, _P,
                                          _P]),
    "kg_sector_dim": (ctypes.c_int, [ctypes.POINTER(KgSector), ctypes.POINTER(ctypes.c_int32)]),
    "kg_sector_states": (ctypes.c_int, [ctypes.POINTER(KgSector), ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32]),
    "kg_sector_apply_h0": (ctypes.c_int, [ctypes.POINTER(KgSector), _P, _P, ctypes.c_int32]),
    "kg_sector_workspace_bytes": (ctypes.c_int, [ctypes.POINTER(KgSector), ctypes.POINTER(KgOptions), ctypes.c_int32,
                                                 ctypes.POINTER(ctypes.c_size_t)]),
    "kg_sector_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(KgSector), ctypes.POINTER(KgOptions),
                                        ctypes.c_int32, _P, ctypes.c_size_t, _P]),
    "kg_sector_evaluate": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "kg_sector_sync": (ctypes.c_int, [_P, ctypes.POINTER(KgReport)]),
    "kg_sector_destroy": (ctypes.c_int, [_P]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """The loaded CUDA library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                               f"g.build()\"` (needs nvcc); the K-GRAPE path has no CPU fallback")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        _lib = handle
    return _lib


class KGrapeError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().kg_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != KG_OK:
        raise KGrapeError(status, where)
