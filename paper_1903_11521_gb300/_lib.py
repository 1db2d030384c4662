"""ctypes binding of the C ABI declared in include/yateto_gb300.h (marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

_LIB = None


class YtError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {message} (status {status})")
        self.status = status


class TensorDesc(C.Structure):
    _fields_ = [("name", C.c_char_p), ("ndim", C.c_int32), ("shape", C.POINTER(C.c_int32)),
                ("pattern", C.POINTER(C.c_uint8)), ("values", C.POINTER(C.c_double))]


class PlanStats(C.Structure):
    _fields_ = [("nz_flops", C.c_double), ("hw_flops", C.c_double), ("naive_flops", C.c_double),
                ("bytes_per_element", C.c_int64), ("n_ops", C.c_int32), ("n_terms", C.c_int32),
                ("log_cost", C.c_int64 * 4), ("order", C.c_char * 1024)]


class MeshDesc(C.Structure):
    _fields_ = [("n_elements", C.c_int64), ("material", C.POINTER(C.c_double)),
                ("jacobian", C.POINTER(C.c_double)), ("neighbours", C.POINTER(C.c_int32)),
                ("faces", C.POINTER(C.c_int8)), ("orient", C.POINTER(C.c_int8)),
                ("attenuation", C.POINTER(C.c_double)), ("n_halo", C.c_int64)]


class SchemeDesc(C.Structure):
    _fields_ = [("order", C.c_int32), ("dt", C.c_double), ("precision", C.c_int),
                ("flags", C.c_int32), ("quantities", C.c_int32)]


class ServerDesc(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("precision", C.c_int), ("flags", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("submitted", "completed", "failed", "pending", "active",
                                         "max_active", "ticks", "budget_bytes", "peak_bytes")] + \
               [("element_updates", C.c_double)]


YT_F64, YT_F32, YT_BF16X3_F32ACC = 0, 1, 2
YT_MEM_HOST, YT_MEM_DEVICE = 0, 1
YT_FIELD_DOFS, YT_FIELD_TIME_INTEGRAL = 0, 1
YT_SCHEME_DIAG_EXPIRE_WAIT = 1

# every symbol declared in include/yateto_gb300.h with its (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "yt_status_string": (C.c_char_p, [C.c_int]),
    "yt_last_error": (C.c_char_p, []),
    "yt_version": (C.c_char_p, []),
    "yt_plan_create": (C.c_int, [C.c_char_p, C.POINTER(TensorDesc), C.c_int32, C.c_int, C.POINTER(_P)]),
    "yt_plan_stats_get": (C.c_int, [_P, C.POINTER(PlanStats)]),
    "yt_plan_eqspp": (C.c_int, [_P, C.c_int32, C.c_int32, C.POINTER(C.c_uint8)]),
    "yt_execute_batched": (C.c_int, [_P, C.POINTER(_P), C.c_int64, _P]),
    "yt_execute_batched_noalloc": (C.c_int, [_P, C.POINTER(_P), C.c_int64, _P]),
    "yt_plan_destroy": (None, [_P]),
    "yt_solver_create": (C.c_int, [C.POINTER(MeshDesc), C.POINTER(SchemeDesc), _P, C.POINTER(_P)]),
    "yt_solver_set_dofs": (C.c_int, [_P, _P, C.c_int, _P]),
    "yt_solver_get": (C.c_int, [_P, C.c_int, _P, C.c_int, _P]),
    "yt_step": (C.c_int, [_P, _P]),
    "yt_step_local": (C.c_int, [_P, _P]),
    "yt_step_neighbour": (C.c_int, [_P, _P]),
    "yt_step_phase": (C.c_int, [_P, C.c_int32, _P]),
    "yt_step_host": (C.c_int, [_P, _P, _P, _P]),
    "yt_solver_stats": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "yt_solver_status": (C.c_int, [_P, _P]),
    "yt_solver_reference_matrix": (C.c_int, [_P, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "yt_solver_destroy": (None, [_P]),
    "yt_solver_set_send_list": (C.c_int, [_P, C.POINTER(C.c_int32), C.c_int64]),
    "yt_solver_halo_pack": (C.c_int, [_P, _P, _P]),
    "yt_solver_halo_buffer": (C.c_int, [_P, C.POINTER(_P), C.POINTER(C.c_int64)]),
    "yt_solver_halo_unpack": (C.c_int, [_P, _P, _P]),
    "yt_step_phase_tiles": (C.c_int, [_P, C.c_int32, C.c_int64, C.c_int64, _P]),
    "yt_batch_create": (C.c_int, [C.POINTER(MeshDesc), C.POINTER(C.c_int8), C.POINTER(SchemeDesc), _P, C.POINTER(_P)]),
    "yt_batch_set_dofs": (C.c_int, [_P, _P, C.c_int, _P]),
    "yt_batch_get": (C.c_int, [_P, C.c_int, _P, C.c_int, _P]),
    "yt_batch_step": (C.c_int, [_P, _P]),
    "yt_batch_tune": (C.c_int, [_P, C.c_int32, _P, C.POINTER(C.c_int32)]),
    "yt_batch_set_form": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32]),
    "yt_batch_config": (C.c_int, [_P, C.c_char_p, C.c_int32]),
    "yt_batch_status": (C.c_int, [_P, _P]),
    "yt_batch_stats": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32)]),
    "yt_batch_destroy": (None, [_P]),
    "yt_server_create": (C.c_int, [C.POINTER(ServerDesc), C.POINTER(_P)]),
    "yt_server_submit": (C.c_int, [_P, C.POINTER(MeshDesc), C.c_int32, C.c_double, _P, C.c_int32,
                                   C.POINTER(C.c_int64)]),
    "yt_server_wait": (C.c_int, [_P, C.c_int64, _P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "yt_server_stats_get": (C.c_int, [_P, C.POINTER(ServerStats)]),
    "yt_server_destroy": (None, [_P]),
    "yt_server_fail_tick": (C.c_int, [_P, C.c_int64]),
    "yt_reference_matrix": (C.c_int, [C.c_int32, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "yt_tc_operands": (C.c_int, [C.c_int32, C.c_int32, _P, C.POINTER(C.c_int64)]),
    "yt_selftest_conversions": (C.c_int, [C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """The loaded shared library.  Raises if it has not been built (there is no fallback)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"{path} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        _build.build()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(status: int, where: str):
    if status != 0:
        lib = load()
        msg = lib.yt_last_error().decode() or lib.yt_status_string(status).decode()
        raise YtError(status, where, msg)
