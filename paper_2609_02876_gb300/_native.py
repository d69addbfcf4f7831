"""ctypes binding of libgradsolve.so (the C-ABI of include/gs.h).

Argument marshalling only. The library must be built (``build.build()``);
there is no fallback: a missing library raises immediately.
"""
from __future__ import annotations

import ctypes as C
import os
import re

from . import build as _build

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_UNKNOWN_PROBLEM, GS_ERR_OOM, GS_ERR_CUDA, GS_ERR_TRAJ_FAILED, \
    GS_ERR_TIMEOUT = range(7)
GS_FP64, GS_FP32_MIXED = 0, 1
GS_CONTROL_FAST, GS_CONTROL_FP64 = 0, 1
GS_METHOD_AUTO, GS_METHOD_TSIT5, GS_METHOD_RODAS5P, GS_METHOD_ROSENBROCK23, GS_METHOD_VERNER7 = 0, 1, 2, 3, 4
PROBLEMS = {"lorenz": 0, "vdp": 1, "robertson": 2, "hires": 3, "linear": 4, "lv_ude": 5, "nrob": 6}
TRAJ_STATUS = {0: "ok", 1: "maxsteps", 2: "dt_underflow", 3: "nonfinite", 4: "singular"}


class GsOptions(C.Structure):
    _fields_ = [("precision", C.c_int), ("method", C.c_int), ("ckpt_k", C.c_int), ("max_steps", C.c_int64),
                ("h0", C.c_double), ("step_counts", C.c_void_p), ("kernel_ms", C.POINTER(C.c_float)),
                ("timeout_ms", C.c_double), ("record_info", C.POINTER(C.c_int32)), ("control", C.c_int),
                ("record_stages", C.c_int)]


class GsError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} (gs_status {code})")


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib():
    """The loaded library. Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2609_02876_gb300.build.build() "
                               "(the CUDA path has no fallback)")
        L = C.CDLL(path)
        vp, i32, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
        L.gs_status_string.argtypes = [i32]
        L.gs_status_string.restype = C.c_char_p
        L.gs_default_options.argtypes = [C.POINTER(GsOptions)]
        L.gs_problem_info.argtypes = [i32, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]
        L.gs_forward_record.argtypes = [i32, i64, vp, vp, vp, d, d, C.POINTER(C.c_double), i32, d, d,
                                        C.POINTER(GsOptions), vp, vp, vp, C.POINTER(vp)]
        L.gs_reverse.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.gs_measure_fma_peak.argtypes = [i32, C.POINTER(C.c_double)]
        L.gs_solve_grad.argtypes = [i32, i64, vp, vp, vp, d, d, C.POINTER(C.c_double), i32, d, d,
                                    C.POINTER(GsOptions), vp, vp, vp, vp, vp, vp]
        L.gs_solve.argtypes = [i32, i64, vp, vp, vp, d, d, C.POINTER(C.c_double), i32, d, d,
                               C.POINTER(GsOptions), vp, vp, vp, vp]
        L.gs_solve_grad_host.argtypes = [i32, i64, vp, vp, vp, d, d, C.POINTER(C.c_double), i32, d, d,
                                         C.POINTER(GsOptions), i64, vp, vp, vp, vp, vp]
        L.gs_record_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.gs_record_stats.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.gs_record_export_mesh.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
        L.gs_record_free.argtypes = [vp]
        L.gs_replay_jvp.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp]
        L.gs_forward_grad.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.gs_record_refresh.argtypes = [vp, vp, vp, vp, vp]
        L.gs_record_refresh.restype = C.c_int
        L.gs_context_create.argtypes = [C.POINTER(vp)]
        L.gs_context_destroy.argtypes = [vp]
        L.gs_context_bytes.argtypes = [vp, C.POINTER(C.c_size_t)]
        L.gs_solve_grad_ctx.argtypes = [vp] + list(L.gs_solve_grad.argtypes)
        for name in ("gs_default_options", "gs_problem_info", "gs_forward_record", "gs_reverse", "gs_solve_grad",
                     "gs_solve", "gs_solve_grad_host", "gs_replay_jvp", "gs_forward_grad",
                     "gs_record_bytes", "gs_record_stats", "gs_record_export_mesh", "gs_record_free",
                     "gs_context_create", "gs_context_destroy", "gs_context_bytes", "gs_solve_grad_ctx"):
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def status_string(code: int) -> str:
    try:
        return lib().gs_status_string(int(code)).decode()
    except RuntimeError:
        return f"status {code}"


def header_symbols(header: str | None = None) -> list[str]:
    """Function names declared in include/gs.h."""
    header = header or os.path.join(_build.ROOT, "include", "gs.h")
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\*]+\s+\**(gs_\w+)\s*\(", text, re.M)))
