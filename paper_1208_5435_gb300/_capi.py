"""ctypes declarations of the C ABI in include/mfipm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmfipm.so")

MFIPM_OK, MFIPM_INVALID_ARG, MFIPM_NOT_CONVERGED, MFIPM_NUMERIC, MFIPM_CUDA, MFIPM_TIMEOUT, MFIPM_UNSUPPORTED = range(7)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "NOT_CONVERGED", 3: "NUMERIC", 4: "CUDA", 5: "TIMEOUT", 6: "UNSUPPORTED"}
OP_DENSE, OP_PARTIAL_DCT, OP_PARTIAL_HAAR = 0, 1, 2
A_F64, A_F32, A_BF16 = 0, 1, 2
PREC_FP64, PREC_FP32_PCG, PREC_BF16_A = 0, 1, 2
OUTER_DF, OUTER_FP64 = 0, 1


class Operator(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("a_dtype", ctypes.c_int32), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("A", ctypes.c_void_p), ("a_scale", ctypes.c_double),
                ("lda", ctypes.c_int64), ("rows", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int32), ("tol_pcg", ctypes.c_double),
                ("max_iter_pcg", ctypes.c_int32), ("sigma1", ctypes.c_double), ("sigma2", ctypes.c_double),
                ("sigma3", ctypes.c_double), ("alpha_bar", ctypes.c_double), ("alpha_tilde", ctypes.c_double),
                ("eta", ctypes.c_double), ("precision", ctypes.c_int32), ("equal_steps", ctypes.c_int32),
                ("cluster_size", ctypes.c_int32), ("outer", ctypes.c_int32), ("outer_f32_gap", ctypes.c_double),
                ("centrality_correctors", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("ipm_iters", ctypes.c_int32), ("correctors", ctypes.c_int32),
                ("pcg_iters", ctypes.c_int32), ("n_mat", ctypes.c_int64), ("rel_gap", ctypes.c_double),
                ("dual_res", ctypes.c_double), ("kkt_rel", ctypes.c_double), ("primal_obj", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class Tuning(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("candidates", ctypes.c_int32), ("cluster_size", ctypes.c_int32),
                ("splits1", ctypes.c_int32), ("splits2", ctypes.c_int32), ("cta_max_n", ctypes.c_int64),
                ("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double), ("stages1", ctypes.c_int32),
                ("stages2", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# Every function the header declares, with its ctypes signature.
_P = ctypes.c_void_p
_PP = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "mfipm_params_default": (ctypes.c_int, [ctypes.POINTER(Params)]),
    "mfipm_workspace_size": (ctypes.c_int, [ctypes.POINTER(Operator), ctypes.c_int32, ctypes.POINTER(Params),
                                            ctypes.POINTER(ctypes.c_size_t)]),
    "mfipm_solve": (ctypes.c_int, [ctypes.POINTER(Operator), _P, ctypes.c_double, ctypes.POINTER(Params), _P, _P, _P,
                                   ctypes.c_size_t, ctypes.POINTER(Info), _P]),
    "mfipm_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(Operator), _P, ctypes.c_double, ctypes.POINTER(Params), _P, _P,
                                           ctypes.POINTER(Info), _P]),
    "mfipm_solve_batched": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Operator), _PP,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(Params), _PP, _PP, _P,
                                           ctypes.c_size_t, ctypes.POINTER(Info), _P]),
    "mfipm_backward": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Operator), _PP, ctypes.POINTER(ctypes.c_double),
                                      _PP, _PP, _PP, _PP, ctypes.POINTER(ctypes.c_double), _PP,
                                      ctypes.POINTER(Params), _P, ctypes.c_size_t, ctypes.POINTER(Info), _P]),
    "mfipm_apply_A": (ctypes.c_int, [ctypes.POINTER(Operator), _P, _P, _P, ctypes.c_size_t, _P]),
    "mfipm_apply_At": (ctypes.c_int, [ctypes.POINTER(Operator), _P, _P, _P, ctypes.c_size_t, _P]),
    "mfipm_kkt_residual": (ctypes.c_int, [ctypes.POINTER(Operator), _P, ctypes.c_double, _P, _P, ctypes.c_size_t,
                                          ctypes.POINTER(ctypes.c_double), _P]),
    "mfipm_last_error": (ctypes.c_char_p, []),
    "mfipm_gemm_bf16": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, _P]),
    "mfipm_set_gemm_mode": (ctypes.c_int, [ctypes.c_int32]),
    "mfipm_fp32_fma_peak": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), _P]),
    "mfipm_set_large_dct_threshold": (ctypes.c_int, [ctypes.c_int64]),
    "mfipm_set_residual_mode": (ctypes.c_int, [ctypes.c_int32]),
    "mfipm_autotune": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(Operator), _PP, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(Params), _PP, _P, ctypes.c_size_t, ctypes.POINTER(Info),
                                      ctypes.POINTER(Tuning), _P]),
    "mfipm_clear_tuning": (ctypes.c_int, []),
    "mfipm_last_operator_stats": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "mfipm_set_timing": (ctypes.c_int, [ctypes.c_int32]),
    "mfipm_last_kernel_ms": (ctypes.c_double, []),
}

_lib = None


class MfipmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"mfipm status {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load libmfipm.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_1208_5435_gb300/build.py "
                              "(the solver has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().mfipm_last_error().decode()


def check(code: int, allow=(MFIPM_OK,)) -> int:
    if code not in allow:
        raise MfipmError(code, last_error())
    return code
