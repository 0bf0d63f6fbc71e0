"""ctypes binding of the C ABI in include/fastvpinn.h (same names).

Argument marshalling only: every step of the loss path runs in the CUDA
library.  If the library is missing the import fails loudly; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfastvpinn.so")

FV_OK, FV_ERR_ARG, FV_ERR_DEGENERATE_ELEMENT, FV_ERR_UNSUPPORTED, FV_ERR_OOM, FV_ERR_CUDA, FV_ERR_TIMEOUT = range(7)
FV_FP64, FV_FP32, FV_TF32, FV_BF16, FV_FP16 = range(5)
FV_G_STORED, FV_G_MATRIX_FREE, FV_G_REGULAR = 0, 1, 2
FV_NORM_TEST, FV_NORM_ELEM = range(2)

ERR_NAMES = {1: "FV_ERR_ARG", 2: "FV_ERR_DEGENERATE_ELEMENT", 3: "FV_ERR_UNSUPPORTED", 4: "FV_ERR_OOM",
             5: "FV_ERR_CUDA", 6: "FV_ERR_TIMEOUT"}


class FVError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (ERR_NAMES.get(code, str(code)), msg))
        self.code = code


class fv_mlp_desc(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("widths", C.POINTER(C.c_int))]


class fv_eval_opts(C.Structure):
    _fields_ = [("mlp_precision", C.c_int), ("eps", C.c_double), ("eps_dev", C.c_void_p), ("bx", C.c_double),
                ("by", C.c_double), ("norm", C.c_int)]


class fv_instance(C.Structure):
    _fields_ = [("mesh", C.c_void_p), ("forcing", C.c_void_p), ("bc", C.c_void_p), ("params_dev", C.c_void_p),
                ("grad_dev", C.c_void_p), ("out_dev", C.c_void_p)]


_vp = C.c_void_p
_pvp = C.POINTER(C.c_void_p)
_dp = C.c_void_p   # host double arrays passed as raw addresses
_i64p = C.POINTER(C.c_int64)

SIGNATURES = {
    "fv_ctx_create": [_pvp, C.c_int, _vp],
    "fv_ctx_set_stream": [_vp, _vp],
    "fv_ctx_destroy": [_vp],
    "fv_last_error": [],
    "fv_ctx_enable_timing": [_vp, C.c_int],
    "fv_ctx_set_activation_stash": [_vp, C.c_int],
    "fv_ctx_kernel_times": [_vp, C.c_int, C.POINTER(C.c_double), _i64p, C.POINTER(C.c_int)],
    "fv_kernel_name": [C.c_int],
    "fv_ctx_reset_kernel_times": [_vp],
    "fv_build_mesh_tensors": [_vp, C.c_int, _dp, C.c_int, _vp, C.c_int, C.c_int, C.c_int, C.c_int, _pvp],
    "fv_mesh_info": [_vp, _i64p],
    "fv_mesh_quad_points": [_vp, _dp],
    "fv_mesh_copy_g": [_vp, _dp],
    "fv_mesh_destroy": [_vp],
    "fv_autotune": [_vp, _vp, C.c_int, _dp],
    "fv_mesh_set_g_mode": [_vp, C.c_int],
    "fv_assemble_forcing": [_vp, _dp, _pvp],
    "fv_forcing_copy": [_vp, _dp],
    "fv_forcing_destroy": [_vp],
    "fv_bc_create": [_vp, C.c_int, _dp, _dp, C.c_double, C.c_int, _dp, _dp, C.c_double, _pvp],
    "fv_bc_destroy": [_vp],
    "fv_loss": [_vp, _vp, _vp, _vp, C.POINTER(fv_mlp_desc), _vp, C.POINTER(fv_eval_opts), _vp],
    "fv_loss_grad": [_vp, _vp, _vp, _vp, C.POINTER(fv_mlp_desc), _vp, C.POINTER(fv_eval_opts), _vp, _vp],
    "fv_loss_grad_noalloc": [_vp, _vp, _vp, _vp, C.POINTER(fv_mlp_desc), _vp, C.POINTER(fv_eval_opts), _vp, _vp],
    "fv_eval_intermediates": [_vp, _vp, _vp, _vp, C.POINTER(fv_mlp_desc), _vp, C.POINTER(fv_eval_opts), _vp, _vp,
                              _vp, _vp],
    "fv_mlp_eval": [_vp, C.POINTER(fv_mlp_desc), _vp, C.c_int, C.c_int, _vp, _vp],
    "fv_adam_create": [_vp, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, _pvp],
    "fv_adam_destroy": [_vp],
    "fv_inverse_step": [_vp, _vp, _vp, _vp, C.POINTER(fv_mlp_desc), _vp, _vp, C.POINTER(fv_eval_opts), _vp,
                        C.c_double, _vp, _vp],
    "fv_step_graph_create": [_vp, _vp, _vp, _vp, C.POINTER(fv_mlp_desc), _vp, _vp, C.POINTER(fv_eval_opts), _vp,
                             C.c_double, _vp, _vp, C.c_int, _pvp],
    "fv_graph_launch": [_vp],
    "fv_graph_destroy": [_vp],
    "fv_batch_plan": [_vp, C.c_int, C.POINTER(fv_instance), C.POINTER(fv_mlp_desc), C.POINTER(fv_eval_opts), C.c_int,
                      _pvp],
    "fv_batch_loss_grad": [_vp],
    "fv_batch_info": [_vp, C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "fv_batch_destroy": [_vp],
}

_lib = None


def lib() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("CUDA library %s is missing: run `python -m paper_2404_12063_b300.build` "
                              "(there is no CPU fallback)" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_char_p if name in ("fv_last_error", "fv_kernel_name") else C.c_int
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != FV_OK:
        raise FVError(rc, lib().fv_last_error().decode())


def call(name: str, *args) -> None:
    check(getattr(lib(), name)(*args))
