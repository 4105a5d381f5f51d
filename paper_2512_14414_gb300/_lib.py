"""ctypes declarations of include/ctm.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libctm.so")

CTM_FP64, CTM_TF32, CTM_BF16, CTM_TF32X3, CTM_BF16X3 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": CTM_FP64, "tf32": CTM_TF32, "bf16": CTM_BF16, "tf32x3": CTM_TF32X3, "bf16x3": CTM_BF16X3}

EXPORTS = ["ctm_create", "ctm_init", "ctm_step", "ctm_energy", "ctm_grad", "ctm_grad_fixed_point", "ctm_get_env", "ctm_set_env",
           "ctm_env_numel", "ctm_kernel_launches", "ctm_set_limits", "ctm_magnetization", "ctm_plaquette_order", "ctm_profile", "ctm_profile_read", "ctm_svd", "ctm_svd_noalloc",
           "ctm_get_spectra", "ctm_mlp_forward", "ctm_mlp_work_floats", "ctm_mlp_backward", "ctm_adam_step", "ctm_destroy", "ctm_error_string"]
PROF_CLASSES = {"gemm": 0, "permute": 1, "svd": 2, "qr": 3, "misc": 4, "tc_gemm": 5, "gemm_f64": 6}


class CtmTerm(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int), ("y", ctypes.c_int), ("kind", ctypes.c_int),
                ("coupling", ctypes.c_double), ("h", ctypes.POINTER(ctypes.c_double))]


class CtmDesc(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("d", ctypes.c_int), ("D", ctypes.c_int),
                ("chi", ctypes.c_int), ("precision", ctypes.c_int), ("n_terms", ctypes.c_int),
                ("terms", ctypes.POINTER(CtmTerm)), ("svd_cutoff_rel", ctypes.c_double),
                ("svd_adjoint_eps", ctypes.c_double), ("max_iter", ctypes.c_int)]


_lib = None


def load():
    """Load libctm.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libctm.so not built ({LIB_PATH}); run paper_2512_14414_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    lib.ctm_create.argtypes = [ctypes.POINTER(CtmDesc), ctypes.POINTER(vp)]
    lib.ctm_init.argtypes = [vp, vp, vp, vp]
    lib.ctm_step.argtypes = [vp, i, ctypes.POINTER(d), vp]
    lib.ctm_energy.argtypes = [vp, vp, vp, vp]
    lib.ctm_grad.argtypes = [vp, i, vp, vp, vp]
    lib.ctm_grad_fixed_point.argtypes = [vp, i, d, vp, vp, ctypes.POINTER(d), vp]
    lib.ctm_get_env.argtypes = [vp, vp, vp]
    lib.ctm_set_env.argtypes = [vp, vp, vp]
    lib.ctm_env_numel.argtypes = [vp]
    lib.ctm_env_numel.restype = i64
    lib.ctm_kernel_launches.argtypes = [vp]
    lib.ctm_kernel_launches.restype = i64
    lib.ctm_set_limits.argtypes = [vp, i, i64]
    lib.ctm_magnetization.argtypes = [vp, vp, vp, vp]
    lib.ctm_plaquette_order.argtypes = [vp, ctypes.POINTER(i), i, ctypes.POINTER(i), i, vp, vp]
    lib.ctm_profile.argtypes = [vp, i]
    lib.ctm_profile_read.argtypes = [vp, i, ctypes.POINTER(d), ctypes.POINTER(i64), ctypes.POINTER(d),
                                     ctypes.POINTER(d)]
    lib.ctm_svd.argtypes = [vp, i, i, vp, vp, vp, vp]
    lib.ctm_svd_noalloc.argtypes = [vp, i, i, vp, vp, vp, vp]
    lib.ctm_get_spectra.argtypes = [vp, i, vp, i, i, ctypes.POINTER(i)]
    lib.ctm_mlp_forward.argtypes = [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, vp]
    lib.ctm_mlp_work_floats.argtypes = [i, i, ctypes.POINTER(i)]
    lib.ctm_mlp_work_floats.restype = i64
    lib.ctm_mlp_backward.argtypes = [vp, vp, i, i, ctypes.POINTER(i), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, vp]
    lib.ctm_adam_step.argtypes = [vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_float, i, vp]
    lib.ctm_destroy.argtypes = [vp]
    lib.ctm_error_string.argtypes = [i]
    lib.ctm_error_string.restype = ctypes.c_char_p
    for f in ("ctm_create", "ctm_init", "ctm_step", "ctm_energy", "ctm_grad", "ctm_get_env", "ctm_set_env",
              "ctm_set_limits", "ctm_magnetization", "ctm_plaquette_order", "ctm_profile", "ctm_profile_read", "ctm_svd", "ctm_svd_noalloc", "ctm_get_spectra", "ctm_mlp_forward",
              "ctm_destroy"):
        getattr(lib, f).restype = i
    _lib = lib
    return lib
