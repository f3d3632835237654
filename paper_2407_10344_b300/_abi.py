"""ctypes declarations of the C ABI in ``include/glim_lin.h`` (argument marshalling only).

The shared library is built in-tree (``paper_2407_10344_b300/libglimlin.so``).  Loading
fails loudly when it is missing: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libglimlin.so")

GLIM_OK = 0
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "EHASHFULL", -5: "ERANGE",
                -6: "ENOTPD", -7: "ETIMEOUT"}
ACC_FP32, ACC_KAHAN, ACC_FP64 = 0, 1, 2
MAX_LEVELS = 4
RECORD_DOUBLES = 92  # GLIM_RECORD_DOUBLES: e, the upper triangle of H (78), b (12), inliers

# every function the header declares, with (restype, argtypes)
_vp, _i32, _i64, _f32, _f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double


class Frame(C.Structure):
    _fields_ = [("pts4", _vp), ("cov6", _vp), ("normal3", _vp), ("n", _i64)]


class Pair(C.Structure):
    _fields_ = [("src_frame", _i32), ("tgt_frame", _i32), ("tgt", _vp)]


class LinOpts(C.Structure):
    _fields_ = [("validate_surface", _i32), ("accum_mode", _i32), ("block", _i32), ("pts_per_thread", _i32),
                ("blocks_per_sm", _i32), ("persistent", _i32), ("kernel", _i32), ("reserved", _i32)]


SIGNATURES = {
    "glim_create": (_i32, [C.POINTER(_vp), C.c_int, _vp]),
    "glim_destroy": (None, [_vp]),
    "glim_last_error": (C.c_char_p, [_vp]),
    "glim_num_sms": (_i32, [_vp]),
    "glim_kernel_launches": (_i64, [_vp]),
    "glim_debug_fail_allocation": (None, [_i64]),
    "glim_fp32_fma_peak": (_i32, [_vp, _i32, C.POINTER(C.c_double)]),
    "glim_fp64_fma_peak": (_i32, [_vp, _i32, C.POINTER(C.c_double)]),
    "glim_estimate_covariances": (_i32, [_vp, _vp, _i64, _i32, _i32, _f32, _vp, _vp]),
    "glim_estimate_covariances_knn": (_i32, [_vp, _vp, _i64, _i32, _i32, _f32, _vp, _vp, _vp]),
    "glim_spatial_order": (_i32, [_vp, _vp, _i64, _f32, _vp]),
    "glim_build_voxelmap": (_i32, [_vp, _vp, _vp, _i64, _vp, _i32, C.POINTER(_vp)]),
    "glim_build_voxelmap_ex": (_i32, [_vp, _vp, _vp, _i64, _vp, _i32, _i32, C.POINTER(_vp)]),
    "glim_vmap_free": (None, [_vp]),
    "glim_vmap_insert": (_i32, [_vp, _vp, _vp, _vp, _i64, _i32]),
    "glim_vmap_is_dense": (_i32, [_vp, _i32]),
    "glim_vmap_info": (_i32, [_vp, _i32, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i32)]),
    "glim_vmap_export": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp, _vp]),
    "glim_correspondences": (_i32, [_vp, C.POINTER(Frame), _vp, _vp, _vp, _i32, _vp]),
    "glim_overlap": (_i32, [_vp, C.POINTER(Frame), _i32, C.POINTER(Pair), _i32, _vp, _i32, _vp]),
    "glim_linearize_factors": (_i32, [_vp, C.POINTER(Frame), _i32, C.POINTER(Pair), _i32, _vp,
                                      C.POINTER(LinOpts), _vp, _vp, _vp, _vp]),
    "glim_linearize_factors_plain": (_i32, [_vp, C.POINTER(Frame), _i32, C.POINTER(Pair), _i32, _vp,
                                            C.POINTER(LinOpts), _vp, _vp, _vp, _vp]),
    "glim_linearize_factors_noalloc": (_i32, [_vp, C.POINTER(Frame), _i32, C.POINTER(Pair), _i32, _vp,
                                              C.POINTER(LinOpts), _vp, _vp, _vp, _vp]),
    "glim_plan_create": (_i32, [_vp, C.POINTER(Frame), _i32, C.POINTER(Pair), _i32, C.POINTER(LinOpts),
                                C.POINTER(_vp)]),
    "glim_plan_destroy": (None, [_vp]),
    "glim_plan_linearize": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "glim_plan_set_poses": (_i32, [_vp, _vp]),
    "glim_plan_relative_poses": (_i32, [_vp, _vp, _vp]),
    "glim_plan_correspondence_ids": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "glim_plan_launch": (_i32, [_vp]),
    "glim_plan_device_outputs": (_i32, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp)]),
    "glim_plan_device_records": (_i32, [_vp, C.POINTER(_vp)]),
    "glim_plan_kernels_per_launch": (_i32, [_vp]),
    "glim_plan_launch_timed": (_i32, [_vp, _i32]),
    "glim_plan_kernel_ms": (_i32, [_vp, _i32, C.POINTER(_f32)]),
    "glim_plan_autotune": (_i32, [_vp, _vp, _i32, C.POINTER(LinOpts), C.POINTER(_f32)]),
    "glim_plan_linearize_pinned": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "glim_plan_get_opts": (_i32, [_vp, C.POINTER(LinOpts)]),
    "glim_backward": (_i32, [_vp, C.POINTER(Frame), _i32, C.POINTER(Pair), _i32, _vp, _i32, _i32, _vp, _vp,
                             _vp]),
    "glim_plan_backward": (_i32, [_vp, _vp, _i32, _vp, _vp, _vp]),
    "glim_plan_gauss_newton": (_i32, [_vp, _vp, _i32, _i32, _vp, _vp, _vp]),
    "glim_gn_solve": (_i32, [_vp, _vp, _i32, _i64, _vp, _i64, _i32, _i64, _vp, _vp]),
    "glim_graph_step": (_i32, [_vp, _vp, _i32, _i32, _vp, _vp, _i32, _f64, _vp, _vp, _vp]),
}

_lib = None


def load():
    """Load the library and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2407_10344_b300.build` (there is no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
