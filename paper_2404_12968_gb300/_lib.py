"""ctypes binding of libgabp.so (include/gabp.h).  Argument marshalling only.

Every step of the GaBP path runs in the library's CUDA kernels; there is no Python or CPU
fallback.  If the shared library has not been built, loading raises immediately.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgabp.so")

GABP_OK = 0
GABP_ERR_ARG = 1
GABP_ERR_OOM = 2
GABP_ERR_CUDA = 3
GABP_ERR_DIVERGED = 4
GABP_ERR_TIMEOUT = 5
GABP_ERR_STATE = 6
GABP_FP32 = 0
GABP_FP64 = 1
GABP_INIT_COLD = 0
GABP_INIT_PAPER = 1
GABP_KERNEL_AUTO = 0
GABP_KERNEL_FUSED = 1
GABP_KERNEL_SPLIT = 2
GABP_KERNEL_TMA = 3
GABP_KERNEL_SWEEP = 4

_ERRNAMES = {1: "GABP_ERR_ARG", 2: "GABP_ERR_OOM", 3: "GABP_ERR_CUDA", 4: "GABP_ERR_DIVERGED",
             5: "GABP_ERR_TIMEOUT", 6: "GABP_ERR_STATE"}


class gabp_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("h", ctypes.c_double)]


class gabp_prior(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("boundary", ctypes.c_int), ("alpha", ctypes.c_int)]


class gabp_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("init", ctypes.c_int), ("kernel", ctypes.c_int),
                ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int), ("tol", ctypes.c_double),
                ("check_every", ctypes.c_int), ("max_iters", ctypes.c_int), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("debug_flags", ctypes.c_int), ("tile_run", ctypes.c_int)]


class gabp_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("last_residual", ctypes.c_double),
                ("n", ctypes.c_int64), ("m", ctypes.c_int64), ("edges", ctypes.c_int64),
                ("precision", ctypes.c_int), ("kernel", ctypes.c_int), ("tile_x", ctypes.c_int),
                ("tile_y", ctypes.c_int), ("bytes_per_iter", ctypes.c_double), ("tile_run", ctypes.c_int)]


MG_MAX_LEVELS = 16


class gabp_mg_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("iterations", ctypes.c_int64 * MG_MAX_LEVELS),
                ("damping", ctypes.c_double * MG_MAX_LEVELS), ("residual", ctypes.c_double * MG_MAX_LEVELS),
                ("converged", ctypes.c_int * MG_MAX_LEVELS)]


class gabp_problem(ctypes.Structure):
    _fields_ = [("grid", gabp_grid), ("kappa", ctypes.c_double), ("gamma", ctypes.c_double),
                ("m", ctypes.c_int64), ("obs_xy", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("noise_var", ctypes.c_void_p)]


class GabpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


_LIB = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


def load():
    """Load libgabp.so; raises if it is missing (no fallback path exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libgabp.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    L.gabp_default_options.argtypes = [ctypes.POINTER(gabp_options)]
    L.gabp_default_options.restype = None
    L.gabp_create.argtypes = [ctypes.POINTER(_vp), gabp_grid, ctypes.c_double,
                              ctypes.POINTER(gabp_prior), ctypes.c_int64, _vp, _vp, _vp,
                              ctypes.POINTER(gabp_options)]
    L.gabp_create.restype = ctypes.c_int
    L.gabp_iterate.argtypes = [_vp, ctypes.c_int, ctypes.c_double]
    L.gabp_iterate.restype = ctypes.c_int
    L.gabp_marginals.argtypes = [_vp, _vp, _vp]
    L.gabp_marginals.restype = ctypes.c_int
    L.gabp_residual.argtypes = [_vp, _dp]
    L.gabp_residual.restype = ctypes.c_int
    L.gabp_pw_create.argtypes = [ctypes.POINTER(_vp), _vp]
    L.gabp_pw_create.restype = ctypes.c_int
    L.gabp_pw_iterate.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.gabp_pw_iterate.restype = ctypes.c_int
    L.gabp_pw_marginals.argtypes = [_vp, _vp, _vp]
    L.gabp_pw_marginals.restype = ctypes.c_int
    L.gabp_pw_residual.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    L.gabp_pw_residual.restype = ctypes.c_int
    L.gabp_pw_reset.argtypes = [_vp]
    L.gabp_pw_reset.restype = ctypes.c_int
    L.gabp_pw_iterations.argtypes = [_vp]
    L.gabp_pw_iterations.restype = ctypes.c_int64
    L.gabp_pw_message_change.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    L.gabp_pw_message_change.restype = ctypes.c_int
    L.gabp_pw_iterate_early_stop.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.POINTER(ctypes.c_int64)]
    L.gabp_pw_iterate_early_stop.restype = ctypes.c_int
    L.gabp_pw_iterate_early_stop_ref.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.POINTER(ctypes.c_double)]
    L.gabp_pw_iterate_early_stop_ref.restype = ctypes.c_int
    L.gabp_pw_upscale.argtypes = [_vp, _vp]
    L.gabp_pw_upscale.restype = ctypes.c_int
    L.gabp_pw_last_error.argtypes = [_vp]
    L.gabp_pw_last_error.restype = ctypes.c_char_p
    L.gabp_pw_destroy.argtypes = [_vp]
    L.gabp_pw_destroy.restype = None
    L.gabp_message_change.argtypes = [_vp, ctypes.POINTER(ctypes.c_double)]
    L.gabp_message_change.restype = ctypes.c_int
    L.gabp_iterate_early_stop.argtypes = [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_int64)]
    L.gabp_iterate_early_stop.restype = ctypes.c_int
    L.gabp_mg_create.argtypes = [ctypes.POINTER(_vp), _vp, ctypes.c_int]
    L.gabp_mg_create.restype = ctypes.c_int
    L.gabp_mg_warm_start.argtypes = [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.POINTER(gabp_mg_stats)]
    L.gabp_mg_warm_start.restype = ctypes.c_int
    L.gabp_mg_last_error.argtypes = [_vp]
    L.gabp_mg_last_error.restype = ctypes.c_char_p
    L.gabp_mg_destroy.argtypes = [_vp]
    L.gabp_mg_destroy.restype = None
    L.gabp_warm_start.argtypes = [_vp, _vp, _vp]
    L.gabp_warm_start.restype = ctypes.c_int
    L.gabp_reset.argtypes = [_vp]
    L.gabp_reset.restype = ctypes.c_int
    L.gabp_message_bytes.argtypes = [_vp]
    L.gabp_message_bytes.restype = ctypes.c_int64
    L.gabp_get_messages.argtypes = [_vp, _vp]
    L.gabp_get_messages.restype = ctypes.c_int
    L.gabp_set_messages.argtypes = [_vp, _vp]
    L.gabp_set_messages.restype = ctypes.c_int
    L.gabp_get_stats.argtypes = [_vp, ctypes.POINTER(gabp_stats)]
    L.gabp_get_stats.restype = ctypes.c_int
    L.gabp_last_error.argtypes = [_vp]
    L.gabp_last_error.restype = ctypes.c_char_p
    L.gabp_create_error.argtypes = []
    L.gabp_create_error.restype = ctypes.c_char_p
    L.gabp_destroy.argtypes = [_vp]
    L.gabp_destroy.restype = None
    L.gabp_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(gabp_problem),
                                    ctypes.POINTER(gabp_options)]
    L.gabp_batch_create.restype = ctypes.c_int
    L.gabp_batch_iterate.argtypes = [_vp, ctypes.c_int, ctypes.c_double]
    L.gabp_batch_iterate.restype = ctypes.c_int
    L.gabp_batch_residuals.argtypes = [_vp, _dp]
    L.gabp_batch_residuals.restype = ctypes.c_int
    L.gabp_batch_marginals.argtypes = [_vp, ctypes.c_int, _vp, _vp]
    L.gabp_batch_marginals.restype = ctypes.c_int
    L.gabp_batch_get_stats.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(gabp_stats)]
    L.gabp_batch_get_stats.restype = ctypes.c_int
    L.gabp_batch_strip_height.argtypes = [_vp]
    L.gabp_batch_strip_height.restype = ctypes.c_int
    L.gabp_batch_last_error.argtypes = [_vp]
    L.gabp_batch_last_error.restype = ctypes.c_char_p
    L.gabp_batch_destroy.argtypes = [_vp]
    L.gabp_batch_destroy.restype = None
    _fp = ctypes.POINTER(ctypes.c_float)
    L.gabp_wsnet_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_uint64, ctypes.c_int]
    L.gabp_wsnet_create.restype = ctypes.c_int
    L.gabp_wsnet_param_count.argtypes = [_vp]
    L.gabp_wsnet_param_count.restype = ctypes.c_int64
    L.gabp_wsnet_get_params.argtypes = [_vp, _vp]
    L.gabp_wsnet_get_params.restype = ctypes.c_int
    L.gabp_wsnet_set_params.argtypes = [_vp, _vp]
    L.gabp_wsnet_set_params.restype = ctypes.c_int
    L.gabp_wsnet_set_kernels.argtypes = [_vp, ctypes.c_int]
    L.gabp_wsnet_set_kernels.restype = ctypes.c_int
    L.gabp_wsnet_forward.argtypes = [_vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]
    L.gabp_wsnet_forward.restype = ctypes.c_int
    L.gabp_wsnet_gradients.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, _vp, _fp]
    L.gabp_wsnet_gradients.restype = ctypes.c_int
    L.gabp_wsnet_train_step.argtypes = [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_float, _fp]
    L.gabp_wsnet_train_step.restype = ctypes.c_int
    L.gabp_wsnet_last_error.argtypes = [_vp]
    L.gabp_wsnet_last_error.restype = ctypes.c_char_p
    L.gabp_wsnet_create_error.argtypes = []
    L.gabp_wsnet_create_error.restype = ctypes.c_char_p
    L.gabp_wsnet_destroy.argtypes = [_vp]
    L.gabp_wsnet_destroy.restype = None
    L.gabp_wsnet_input_shape.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]
    L.gabp_wsnet_input_shape.restype = ctypes.c_int
    L.gabp_wsnet_sample.argtypes = [_vp, _vp, _vp]
    L.gabp_wsnet_sample.restype = ctypes.c_int
    L.gabp_batch_input_shape.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), _dp]
    L.gabp_batch_input_shape.restype = ctypes.c_int
    L.gabp_batch_wsnet_sample.argtypes = [_vp, ctypes.c_int, _vp, _vp]
    L.gabp_batch_wsnet_sample.restype = ctypes.c_int
    L.gabp_wsnet_warm_start.argtypes = [_vp, _vp]
    L.gabp_wsnet_warm_start.restype = ctypes.c_int
    L.gabp_set_prior_mean.argtypes = [_vp, _vp]
    L.gabp_set_prior_mean.restype = ctypes.c_int
    L.gabp_residual_noalloc.argtypes = [gabp_grid, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                        _vp, _vp, _vp, _vp, _dp, _vp]
    L.gabp_residual_noalloc.restype = ctypes.c_int
    L.gabp_residual_noalloc_error.argtypes = []
    L.gabp_residual_noalloc_error.restype = ctypes.c_char_p
    _LIB = L
    return L
