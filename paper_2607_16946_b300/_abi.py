"""ctypes view of include/ptsdf.h (libptsdf.so).  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.

Importing this module loads the in-tree libptsdf.so and raises if it is
missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libptsdf.so")

SDF_OK, SDF_EINVAL, SDF_ENOMEM, SDF_ECUDA, SDF_EBUSY, SDF_ETIMEOUT, SDF_EDEVICE = range(7)
SDF_F32, SDF_F16X2, SDF_BF16X2 = 0, 1, 2
SDF_LAMBDA_GLOBAL, SDF_LAMBDA_FIXED, SDF_LAMBDA_RADIUS = 0, 1, 2
SDF_RADIUS_FALLBACK_K = 32
SDF_ENGINE_AUTO, SDF_ENGINE_ALU, SDF_ENGINE_TENSOR = 0, 1, 2
SDF_FORMULA_BLEND, SDF_FORMULA_LSE, SDF_FORMULA_SSPD, SDF_FORMULA_SHC = 0, 1, 2, 3
SDF_DEV_WAIT_TIMEOUT, SDF_DEV_BAD_INPUT = 1, 2
SDF_K_PREPASS, SDF_K_FWD, SDF_K_MERGE, SDF_K_BUILD, SDF_K_FWD_GRAD, SDF_K_BWD, SDF_K_FWD_TC = 0, 1, 2, 3, 4, 5, 6
SDF_K_RADIUS, SDF_K_KNN, SDF_K_PLANE = 7, 8, 9
SDF_UNION, SDF_INTERSECT, SDF_DIFFERENCE = 0, 1, 2
KERNEL_IDS = {"prepass": 0, "fwd": 1, "merge": 2, "build": 3, "fwd_grad": 4, "bwd_params": 5, "fwd_tc": 6,
              "radius": 7, "knn": 8, "plane": 9}

STATUS_NAMES = {0: "SDF_OK", 1: "SDF_EINVAL", 2: "SDF_ENOMEM", 3: "SDF_ECUDA", 4: "SDF_EBUSY",
                5: "SDF_ETIMEOUT", 6: "SDF_EDEVICE"}


class SdfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class sdf_query_opts(ctypes.Structure):
    _fields_ = [("lambda_mode", ctypes.c_int32), ("precision", ctypes.c_int32), ("C", ctypes.c_float),
                ("fixed_lambda", ctypes.c_float), ("offset", ctypes.c_float), ("split_n", ctypes.c_int32),
                ("engine", ctypes.c_int32), ("formula", ctypes.c_int32)]


# (name, restype, argtypes) for every entry point of include/ptsdf.h
_P, _I64, _I32, _F = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
SIGNATURES = {
    "sdf_opts_default": (ctypes.c_int, [ctypes.POINTER(sdf_query_opts)]),
    "sdf_probe_rates": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "sdf_probe_timing": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "sdf_selftest_soft_sqrt": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "sdf_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                                 ctypes.POINTER(ctypes.c_double)]),
    "sdf_orient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_int32, ctypes.POINTER(sdf_query_opts), ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int32), ctypes.c_void_p]),
    "sdf_query_laplacian": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(sdf_query_opts),
                                           ctypes.c_void_p]),
    "sdf_mesh_level_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                          ctypes.c_float, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p]),
    "sdf_knn_mean_distance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                             ctypes.c_void_p]),
    "sdf_paper_lambda": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "sdf_build": (ctypes.c_int, [_P, _P, _P, _I64, _P, ctypes.POINTER(_P)]),
    "sdf_build_weighted": (ctypes.c_int, [_P, _P, _P, _P, _I64, _P, ctypes.POINTER(_P)]),
    "sdf_project_level_set": (ctypes.c_int, [_P, _P, _I64, ctypes.c_float, ctypes.c_int32, ctypes.c_float, _P, _P,
                                             _P, ctypes.POINTER(sdf_query_opts), _P]),
    "sdf_destroy": (ctypes.c_int, [_P]),
    "sdf_export": (ctypes.c_int, [_P, _P, _I64, ctypes.POINTER(_I64)]),
    "sdf_import": (ctypes.c_int, [_P, _I64, _P, ctypes.POINTER(_P)]),
    "sdf_cloud_info": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_F), ctypes.POINTER(_I64),
                                      ctypes.POINTER(_I64)]),
    "sdf_cloud_forms": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "sdf_query": (ctypes.c_int, [_P, _P, _I64, _P, ctypes.POINTER(sdf_query_opts), _P]),
    "sdf_query_host": (ctypes.c_int, [_P, _P, _I64, _P, ctypes.POINTER(sdf_query_opts), _P]),
    "sdf_query_noalloc": (ctypes.c_int, [_P, _P, _I64, _P, ctypes.POINTER(sdf_query_opts), _P]),
    "sdf_query_grad": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, ctypes.POINTER(sdf_query_opts), _P]),
    "sdf_backward_params": (ctypes.c_int, [_P, _P, _I64, _P, _P, _P, ctypes.POINTER(sdf_query_opts), _P]),
    "sdf_trace": (ctypes.c_int, [_P, _P, _P, _I64, _I32, _F, _F, _P, _P, _P, ctypes.POINTER(sdf_query_opts), _P]),
    "sdf_combine": (ctypes.c_int, [_I32, _P, _P, _I64, _P, _P]),
    "sdf_device_status": (ctypes.c_int, [_P, _P, ctypes.POINTER(_I32)]),
    "sdf_serve_create": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
    "sdf_serve_register": (ctypes.c_int, [_P, _P, ctypes.POINTER(_I32)]),
    "sdf_serve_submit": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "sdf_serve_poll": (ctypes.c_int, [_P, ctypes.c_uint64, _I64, _P]),
    "sdf_serve_stats": (ctypes.c_int, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I64)]),
    "sdf_serve_shutdown": (ctypes.c_int, [_P]),
    "sdf_profile_enable": (ctypes.c_int, [_I32]),
    "sdf_profile_read": (ctypes.c_int, [_I32, ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_double)]),
    "sdf_kernel_name": (ctypes.c_char_p, [_I32]),
    "sdf_last_error": (ctypes.c_char_p, []),
    "sdf_version": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded library (raises FileNotFoundError / OSError if it is absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise FileNotFoundError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2607_16946_b300.build` "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(status: int, what: str = ""):
    if status != SDF_OK:
        msg = lib().sdf_last_error().decode(errors="replace")
        raise SdfError(status, f"{what}: {msg}" if what else msg)


def make_opts(C: float = 64.0, lambda_mode: int = SDF_LAMBDA_GLOBAL, fixed_lambda: float = 0.0,
              offset: float = 0.0, split_n: int = 0, precision: int = SDF_F32,
              engine: int = SDF_ENGINE_AUTO, formula: int = SDF_FORMULA_BLEND) -> sdf_query_opts:
    o = sdf_query_opts()
    check(lib().sdf_opts_default(ctypes.byref(o)))
    o.C, o.lambda_mode, o.fixed_lambda, o.offset, o.split_n, o.precision, o.engine, o.formula = (
        float(C), int(lambda_mode), float(fixed_lambda), float(offset), int(split_n), int(precision), int(engine),
        int(formula))
    return o
