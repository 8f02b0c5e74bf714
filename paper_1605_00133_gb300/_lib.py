"""ctypes binding of libpat.so (include/pat.h).  Argument marshalling only: every step of A, A^T and
C runs in the library's CUDA kernels.  There is no CPU fallback; if the library is missing or the
device is unusable, calls raise."""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpat.so")

PAT_OK = 0
STATUS_NAMES = {0: "PAT_OK", 1: "PAT_ERR_INVALID_ARG", 2: "PAT_ERR_CUDA", 3: "PAT_ERR_OOM",
                4: "PAT_ERR_TIMEOUT", 5: "PAT_ERR_NOT_CONVERGED", 6: "PAT_ERR_UNSUPPORTED"}

# every symbol include/pat.h declares
EXPORTS = ["pat_create_grid", "pat_destroy_grid", "pat_grid_info", "pat_workspace_bytes",
           "pat_forward", "pat_adjoint", "pat_sample", "pat_sample_adjoint", "pat_profile_enable",
           "pat_profile_read", "pat_last_error", "pat_version", "pat_forward_noalloc", "pat_tv_prox",
           "pat_bregman_solve", "pat_get_indices", "pat_device_status", "pat_debug_copy_fault",
           "pat_set_workspace_limit", "pat_bp_tv"]
# include/pat_unet.h (learned warm start)
UNET_EXPORTS = ["pat_unet_conv3", "pat_unet_wgrad_scratch", "pat_unet_conv3_wgrad", "pat_unet_cast_weights",
                "pat_unet_relu_bwd", "pat_unet_pool", "pat_unet_pool_bwd_add", "pat_unet_up", "pat_unet_up_bwd",
                "pat_unet_input", "pat_unet_head", "pat_unet_head_scratch", "pat_unet_head_bwd", "pat_unet_adam",
                "pat_unet_device_status", "pat_unet_debug_copy_fault"]


class PatError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("nz", ctypes.c_int32), ("ny", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("dx", ctypes.c_double), ("c", ctypes.c_double), ("rho0", ctypes.c_double),
                ("cfl", ctypes.c_double), ("dt", ctypes.c_double), ("T", ctypes.c_int32),
                ("pml_size", ctypes.c_int32), ("pml_alpha", ctypes.c_double),
                ("sensor_z", ctypes.c_int32), ("batch", ctypes.c_int32)]


class SamplingDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("m", ctypes.c_int32),
                ("indices", ctypes.POINTER(ctypes.c_int32)), ("perm", ctypes.POINTER(ctypes.c_int32)),
                ("rows", ctypes.POINTER(ctypes.c_int32))]


class SolveParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("outer", ctypes.c_int32), ("inner", ctypes.c_int32),
                ("prox_iters", ctypes.c_int32), ("L", ctypes.c_double), ("power_iters", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("step_scale", ctypes.c_double),
                ("max_backtrack", ctypes.c_int32), ("stall", ctypes.c_int32),
                ("b_in", ctypes.c_void_p), ("b_out", ctypes.c_void_p)]


class SolveReport(ctypes.Structure):
    _fields_ = [("L", ctypes.c_double), ("inner_total", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("energy", ctypes.c_double), ("n_residual", ctypes.c_int32),
                ("residual", ctypes.c_double * 64)]


_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load libpat.so from the package directory (built by paper_1605_00133_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1605_00133_gb300.build` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        L.pat_create_grid.argtypes = [ctypes.POINTER(GridDesc), ctypes.POINTER(SamplingDesc),
                                      ctypes.POINTER(vp)]
        L.pat_create_grid.restype = ctypes.c_int
        L.pat_destroy_grid.argtypes = [vp]
        L.pat_destroy_grid.restype = None
        L.pat_grid_info.argtypes = [vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double)]
        L.pat_grid_info.restype = ctypes.c_int
        L.pat_workspace_bytes.argtypes = [vp]
        L.pat_workspace_bytes.restype = ctypes.c_int64
        for name in ("pat_forward", "pat_adjoint", "pat_forward_noalloc"):
            fn = getattr(L, name)
            fn.argtypes = [vp, vp, vp, vp]
            fn.restype = ctypes.c_int
        for name in ("pat_sample", "pat_sample_adjoint"):
            fn = getattr(L, name)
            fn.argtypes = [vp, vp, vp, ctypes.c_int32, vp]
            fn.restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int32)
        L.pat_get_indices.argtypes = [vp, ip, ip]
        L.pat_get_indices.restype = ctypes.c_int
        L.pat_tv_prox.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, vp]
        L.pat_tv_prox.restype = ctypes.c_int
        L.pat_bp_tv.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int32, vp]
        L.pat_bp_tv.restype = ctypes.c_int
        L.pat_bregman_solve.argtypes = [vp, vp, vp, vp, ctypes.POINTER(SolveParams),
                                        ctypes.POINTER(SolveReport), vp]
        L.pat_bregman_solve.restype = ctypes.c_int
        L.pat_device_status.argtypes = [vp, vp]
        L.pat_device_status.restype = ctypes.c_int
        L.pat_debug_copy_fault.argtypes = [vp, ctypes.c_int32, ctypes.c_int32]
        L.pat_debug_copy_fault.restype = ctypes.c_int
        L.pat_set_workspace_limit.argtypes = [ctypes.c_int64]
        L.pat_set_workspace_limit.restype = ctypes.c_int
        L.pat_profile_enable.argtypes = [vp, ctypes.c_int32]
        L.pat_profile_enable.restype = ctypes.c_int
        L.pat_profile_read.argtypes = [vp, ctypes.c_int32, ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
        L.pat_profile_read.restype = ctypes.c_int
        i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        L.pat_unet_conv3.argtypes = [vp, i32, i32, vp, i32, vp, i32, i32, i32, i32, i32, vp]
        L.pat_unet_wgrad_scratch.argtypes = [i32, i32, i32, i32, i32]
        L.pat_unet_wgrad_scratch.restype = i64
        L.pat_unet_conv3_wgrad.argtypes = [vp, i32, i32, vp, i32, i32, i32, i32, i32, vp, vp, vp]
        L.pat_unet_cast_weights.argtypes = [vp, i32, i32, vp, vp, vp]
        L.pat_unet_relu_bwd.argtypes = [vp, i32, vp, i32, i32, i64, vp]
        L.pat_unet_pool.argtypes = [vp, i32, i32, i32, i32, i32, vp, i32, vp]
        L.pat_unet_pool_bwd_add.argtypes = [vp, i32, i32, i32, i32, i32, vp, i32, vp]
        L.pat_unet_up.argtypes = [vp, i32, i32, i32, i32, i32, vp, i32, vp]
        L.pat_unet_up_bwd.argtypes = [vp, i32, i32, i32, i32, i32, vp, i32, vp]
        L.pat_unet_input.argtypes = [vp, f32, i64, vp, vp]
        L.pat_unet_head.argtypes = [vp, vp, i64, vp, vp]
        L.pat_unet_head_scratch.argtypes = [i64]
        L.pat_unet_head_scratch.restype = i64
        L.pat_unet_head_bwd.argtypes = [vp, vp, vp, vp, i64, vp, vp, vp, vp, vp]
        L.pat_unet_adam.argtypes = [vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp]
        L.pat_unet_device_status.argtypes = [vp]
        L.pat_unet_debug_copy_fault.argtypes = [i32, i32]
        for name in UNET_EXPORTS:
            if name not in ("pat_unet_wgrad_scratch", "pat_unet_head_scratch"):
                getattr(L, name).restype = ctypes.c_int
        L.pat_last_error.argtypes = []
        L.pat_last_error.restype = ctypes.c_char_p
        L.pat_version.argtypes = []
        L.pat_version.restype = ctypes.c_char_p
        _lib = L
        return L


def check(status: int) -> None:
    if status != PAT_OK:
        msg = load().pat_last_error().decode(errors="replace")
        raise PatError(status, msg)
