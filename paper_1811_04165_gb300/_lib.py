"""Loads libsps.so and declares its C signatures (see include/sps.h).

Raises ImportError when the library has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# SPS_BUILD=checked loads the bounds-checked build (libsps_checked.so, built by
# `python -m paper_1811_04165_gb300.build --checked`); the default is libsps.so.
_PATH = os.path.join(_PKG, "libsps_checked.so" if os.environ.get("SPS_BUILD") == "checked" else "libsps.so")
_lib = None

# every exported entry point with (restype, argtypes)
_P = ctypes.c_void_p
_I32, _I64, _SZ = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
SIGNATURES = {
    "sps_plan_create": (_I32, [_P, _P]),
    "sps_plan_destroy": (_I32, [_P]),
    "sps_plan_input_samples": (_I64, [_P]),
    "sps_plan_step1_samples": (_I64, [_P]),
    "sps_plan_delay_table": (_I32, [_P, _P]),
    "sps_plan_subband_tables": (_I32, [_P, _P, _P]),
    "sps_plan_workspace_bytes": (_I32, [_P, _P]),
    "sps_plan_get_config": (_I32, [_P, _P]),
    "sps_plan_set_config": (_I32, [_P, _P]),
    "sps_dedisperse": (_I32, [_P, _P, _I64, _P, _P, _SZ, _P]),
    "sps_dedisperse_noalloc": (_I32, [_P, _P, _I64, _P, _P]),
    "sps_subband_step1": (_I32, [_P, _P, _I64, _P, _P, _SZ, _P]),
    "sps_subband_step2": (_I32, [_P, _P, _P, _P]),
    "sps_integrate": (_I32, [_P, _P, _P, _P]),
    "sps_snr": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "sps_search": (_I32, [_P, _P, _I64, _P, _P, _SZ, _P, _P, _P, _P, _P]),
    "sps_search_host": (_I32, [_P, _P, _I64, _P, _P, _P, _SZ, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "sps_plan_status": (_I32, [_P, _P, _I32]),
    "sps_plan_check_wait_timeout": (_I32, [_P, _I32, _P]),
    "sps_presum_tables_verify": (_I32, [_P, _I32, _I32, _I32, _I32, _I32, _P]),
    "sps_batch_workspace_bytes": (_I32, [_P, _I32, _I32, _P]),
    "sps_batch_create": (_I32, [_P, _P, _I32, _I32, _P, _SZ, _P]),
    "sps_batch_launch": (_I32, [_P, _P]),
    "sps_batch_destroy": (_I32, [_P]),
    "sps_batch_list_launches": (_I32, [_P, _P]),
    "sps_server_create": (_I32, [_P, _P]),
    "sps_server_add_beam": (_I32, [_P, _P, _P]),
    "sps_server_submit": (_I32, [_P, _I32, _P, _I64, _P, _P, ctypes.c_uint64]),
    "sps_server_remove_beam": (_I32, [_P, _I32]),
    "sps_server_poll": (_I32, [_P, _P, _P, _P, _I32, _P]),
    "sps_server_get_stats": (_I32, [_P, _P]),
    "sps_server_pending": (_I32, [_P, _P]),
    "sps_server_clock": (ctypes.c_double, []),
    "sps_server_destroy": (_I32, [_P]),
    "sps_measure_int_add_rate": (_I32, [_P, _P]),
    "sps_optimize": (_I32, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "sps_tune_space": (_I32, [_P, _I32, _I32, _P, _P, _P, _P]),
    "sps_tune_config": (_I32, [_P, _I32, _P, _P]),
    "sps_tune": (_I32, [_P, _I32, _P, _P, _I64, _P, _P, _SZ, _P, _P, _P, _I32, ctypes.c_double, _P, _P, _P,
                        _P, _P]),
    "sps_status_string": (ctypes.c_char_p, [_I32]),
    "sps_last_error": (ctypes.c_char_p, []),
    "sps_abi_version": (_I32, []),
}


class SpsError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {message} (status {status})")
        self.status = status


def lib_path() -> str:
    return _PATH


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_PATH):
            raise ImportError(
                f"{_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
                "(nvcc for sm_103a); there is no CPU fallback")
        L = ctypes.CDLL(_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(status: int, where: str):
    if status != 0:
        L = lib()
        msg = L.sps_last_error().decode() or L.sps_status_string(status).decode()
        raise SpsError(status, where, msg)
