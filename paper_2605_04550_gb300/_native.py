"""ctypes declarations of the libpsa C ABI (include/psa.h). Marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

from .build import LIB

PSA_OK = 0
PSA_EINVAL = -1
PSA_EWORKSPACE = -2
PSA_ECUDA = -3
PSA_EUNSUPPORTED = -4
PSA_ESTATIC = -5
STATIC_SCRATCH_BYTES = 64 << 20

PT_OK, PT_SINGULAR, PT_NOT_CONVERGED, PT_NONFINITE, PT_NOT_EVALUATED, PT_UNDERFLOW = 0, 1, 2, 3, 4, 5

#: every symbol include/psa.h declares
EXPORTS = (
    "psa_version",
    "psa_strerror",
    "psa_default_opts",
    "psa_workspace_bytes",
    "psa_default_points_in_flight",
    "psa_sigma_min",
    "psa_sigma_min_static",
    "psa_grad_workspace_bytes",
    "psa_sigma_min_grad",
    "psa_sigma_min_pairs",
    "psa_band_grad_from_pairs",
    "psa_contour_init",
    "psa_contour_step",
    "psa_batch_plan_bytes",
    "psa_batch_plan",
    "psa_batch_workspace_bytes",
    "psa_sigma_min_batched",
    "psa_gemm_bf16",
    "psa_mlp_workspace_bytes",
    "psa_mlp_forward",
    "psa_mlp_train_step",
    "psa_mlp_timeouts",
    "psa_dual_workspace_bytes",
    "psa_dual_forward",
    "psa_dual_train_step",
    "psa_matrix_stats",
    "psa_global_features",
    "psa_point_features",
    "psa_point_set_stats",
    "psa_point_features_set",
    "psa_region",
    "psa_tile_slots",
    "psa_probe_dfma_rate",
    "psa_probe_fp64",
)

SYMBOL_SAMPLES, STATS, GLOBAL_FEATURES = 256, 24, 28

MLP_IN, MLP_HIDDEN, MLP_PARAMS = 128, 256, 164865
DUAL_PARAMS, DUAL_TRAINABLE = 115585, 60097

BATCH_ORDER_AUTO, BATCH_ORDER_PLAN, BATCH_ORDER_ESTIMATE = 0, 1, 2


class PsaBand(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("kl", ctypes.c_int32), ("ku", ctypes.c_int32),
                ("bands", ctypes.c_void_p)]


class PsaGrid(ctypes.Structure):
    _fields_ = [("re_min", ctypes.c_double), ("re_max", ctypes.c_double),
                ("im_min", ctypes.c_double), ("im_max", ctypes.c_double),
                ("nx", ctypes.c_int32), ("ny", ctypes.c_int32)]


class PsaLanczosOpts(ctypes.Structure):
    _fields_ = [("k_min", ctypes.c_int32), ("k_max", ctypes.c_int32),
                ("tol", ctypes.c_double), ("seed", ctypes.c_uint64)]


class PsaBatchEntry(ctypes.Structure):
    _fields_ = [("A", PsaBand), ("g", PsaGrid), ("out_offset", ctypes.c_int64)]


class PsaError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libpsa.so; raises if it has not been built (there is no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libpsa.so not found at {path}: build it first "
                               "(python -m paper_2605_04550_gb300.build)")
        lib = ctypes.CDLL(path)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.psa_version.restype = ctypes.c_int
        lib.psa_version.argtypes = []
        lib.psa_strerror.restype = ctypes.c_char_p
        lib.psa_strerror.argtypes = [ctypes.c_int]
        lib.psa_default_opts.restype = PsaLanczosOpts
        lib.psa_default_opts.argtypes = []
        lib.psa_workspace_bytes.restype = ctypes.c_int
        lib.psa_workspace_bytes.argtypes = [ctypes.POINTER(PsaBand), ctypes.POINTER(PsaLanczosOpts), i64, i64,
                                            ctypes.POINTER(ctypes.c_size_t)]
        lib.psa_default_points_in_flight.restype = ctypes.c_int
        lib.psa_default_points_in_flight.argtypes = [ctypes.POINTER(PsaBand), i64, ctypes.POINTER(i64)]
        lib.psa_sigma_min.restype = ctypes.c_int
        lib.psa_sigma_min.argtypes = [ctypes.POINTER(PsaBand), ctypes.POINTER(PsaGrid),
                                      ctypes.POINTER(dbl), i32, vp, i64, vp, vp, vp, vp,
                                      ctypes.POINTER(PsaLanczosOpts), vp, ctypes.c_size_t, vp]
        lib.psa_sigma_min_static.restype = ctypes.c_int
        lib.psa_sigma_min_static.argtypes = [ctypes.POINTER(PsaBand), ctypes.POINTER(PsaGrid),
                                             ctypes.POINTER(dbl), i32, vp, i64, vp, vp, vp, vp,
                                             ctypes.POINTER(PsaLanczosOpts), vp]
        lib.psa_grad_workspace_bytes.restype = ctypes.c_int
        lib.psa_grad_workspace_bytes.argtypes = [ctypes.POINTER(PsaBand), ctypes.POINTER(PsaLanczosOpts), i64,
                                                 ctypes.POINTER(ctypes.c_size_t)]
        lib.psa_sigma_min_grad.restype = ctypes.c_int
        lib.psa_sigma_min_grad.argtypes = [ctypes.POINTER(PsaBand), vp, i64, vp, vp, vp, vp, vp, vp,
                                           ctypes.POINTER(PsaLanczosOpts), vp, ctypes.c_size_t, vp]
        lib.psa_sigma_min_pairs.restype = ctypes.c_int
        lib.psa_sigma_min_pairs.argtypes = [ctypes.POINTER(PsaBand), vp, i64, vp, vp, vp, vp, vp, vp,
                                            ctypes.POINTER(PsaLanczosOpts), vp, ctypes.c_size_t, vp]
        lib.psa_band_grad_from_pairs.restype = ctypes.c_int
        lib.psa_band_grad_from_pairs.argtypes = [ctypes.POINTER(PsaBand), i64, vp, vp, vp, vp, vp]
        lib.psa_contour_init.restype = ctypes.c_int
        lib.psa_contour_init.argtypes = [i32, vp, vp, ctypes.POINTER(PsaGrid), vp, vp, dbl] + [vp] * 8 + [vp]
        lib.psa_contour_step.restype = ctypes.c_int
        lib.psa_contour_step.argtypes = [i32, vp, vp, vp, dbl, dbl] + [vp] * 8 + [vp]
        lib.psa_batch_plan_bytes.restype = ctypes.c_int
        lib.psa_batch_plan_bytes.argtypes = [i32, ctypes.POINTER(ctypes.c_size_t)]
        lib.psa_batch_plan.restype = ctypes.c_int
        lib.psa_batch_plan.argtypes = [ctypes.POINTER(PsaBatchEntry), i32, vp, ctypes.c_size_t]
        lib.psa_batch_workspace_bytes.restype = ctypes.c_int
        lib.psa_batch_workspace_bytes.argtypes = [vp, ctypes.POINTER(PsaLanczosOpts), i64, i32,
                                                  ctypes.POINTER(ctypes.c_size_t)]
        lib.psa_sigma_min_batched.restype = ctypes.c_int
        lib.psa_sigma_min_batched.argtypes = [vp, vp, ctypes.POINTER(dbl), i32, vp, vp, vp, vp,
                                              ctypes.POINTER(PsaLanczosOpts), i64, i32, vp, ctypes.c_size_t, vp,
                                              ctypes.POINTER(vp), i32]
        f32 = ctypes.c_float
        lib.psa_gemm_bf16.restype = ctypes.c_int
        lib.psa_gemm_bf16.argtypes = [vp, i64, vp, i64, i32, i32, i32, vp, i64, vp]
        lib.psa_mlp_workspace_bytes.restype = ctypes.c_int
        lib.psa_mlp_workspace_bytes.argtypes = [i64, i32, ctypes.POINTER(ctypes.c_size_t)]
        lib.psa_mlp_forward.restype = ctypes.c_int
        lib.psa_mlp_forward.argtypes = [vp, vp, i64, vp, vp, ctypes.c_size_t, vp]
        lib.psa_mlp_train_step.restype = ctypes.c_int
        lib.psa_mlp_train_step.argtypes = [vp, vp, vp, i32, f32, vp, vp, i64, vp, vp, ctypes.c_size_t, vp]
        lib.psa_dual_workspace_bytes.restype = ctypes.c_int
        lib.psa_dual_workspace_bytes.argtypes = [i64, i32, ctypes.POINTER(ctypes.c_size_t)]
        lib.psa_dual_forward.restype = ctypes.c_int
        lib.psa_dual_forward.argtypes = [vp, vp, i64, vp, vp, ctypes.c_size_t, vp]
        lib.psa_dual_train_step.restype = ctypes.c_int
        lib.psa_dual_train_step.argtypes = [vp, vp, vp, i32, f32, vp, vp, i64, vp, vp, ctypes.c_size_t, vp]
        lib.psa_mlp_timeouts.restype = ctypes.c_int
        lib.psa_mlp_timeouts.argtypes = [ctypes.POINTER(ctypes.c_uint32)]
        lib.psa_matrix_stats.restype = ctypes.c_int
        lib.psa_matrix_stats.argtypes = [ctypes.POINTER(PsaBand), vp, vp, vp]
        lib.psa_global_features.restype = ctypes.c_int
        lib.psa_global_features.argtypes = [vp, vp, dbl, vp, vp]
        lib.psa_point_features.restype = ctypes.c_int
        lib.psa_point_features.argtypes = [ctypes.POINTER(PsaGrid), vp, i64, vp, vp, vp, vp, vp]
        lib.psa_point_set_stats.restype = ctypes.c_int
        lib.psa_point_set_stats.argtypes = [vp, i32, vp, vp]
        lib.psa_point_features_set.restype = ctypes.c_int
        lib.psa_point_features_set.argtypes = [ctypes.POINTER(PsaGrid), vp, i64, vp, vp, i32, i32, vp, vp, vp]
        lib.psa_region.restype = ctypes.c_int
        lib.psa_region.argtypes = [vp, ctypes.c_float, i32, i32, i32, vp, vp]
        lib.psa_tile_slots.restype = ctypes.c_int
        lib.psa_tile_slots.argtypes = [vp, i32, i32, vp, vp]
        lib.psa_probe_dfma_rate.restype = ctypes.c_int
        lib.psa_probe_dfma_rate.argtypes = [i32, ctypes.POINTER(dbl), vp]
        lib.psa_probe_fp64.restype = ctypes.c_int
        lib.psa_probe_fp64.argtypes = [i32, i32, i32, i32, i32, ctypes.POINTER(dbl), vp]
        _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().psa_strerror(code).decode()
    except Exception:  # pragma: no cover - library missing
        return "unknown"


def check(code: int, what: str) -> None:
    if code != PSA_OK:
        raise PsaError(code, what)
