"""ctypes declarations of the C ABI in ``include/vgpdf.h`` (``libvgpdf.so``).

Loading fails loudly when the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvgpdf.so")

VGP_OK = 0
ERRORS = {-1: "VGP_ERR_ARG", -2: "VGP_ERR_OOM", -3: "VGP_ERR_CUDA", -4: "VGP_ERR_TABLE_FULL",
          -5: "VGP_ERR_TIMEOUT", -6: "VGP_ERR_STATE"}
VGP_FP64, VGP_MIXED = 0, 1
VGP_FUSE_INVVAR, VGP_FUSE_TSDF = 0, 1
VGP_LAUNCH_BATCHED, VGP_LAUNCH_PER_INSTANCE, VGP_LAUNCH_GRAPH = 0, 1, 2
ST_OK, ST_NO_SUPPORT, ST_CLAMPED, ST_BAD_INPUT, ST_FACTOR_FAIL = 0, 1, 2, 3, 4


class VgpParams(C.Structure):
    _fields_ = [("voxel_size", C.c_double), ("lengthscale", C.c_double), ("sigma_occ", C.c_double),
                ("d_max", C.c_double), ("d_var_floor", C.c_double), ("max_pts_leaf", C.c_int32),
                ("max_pts_group", C.c_int32), ("max_leaf_search", C.c_int32), ("fusion", C.c_int32),
                ("precision", C.c_int32), ("profile", C.c_int32), ("launch", C.c_int32), ("normal_steps", C.c_int32),
                ("sigma_prop", C.c_double), ("n_props", C.c_int32), ("emulate_fp64", C.c_int32)]


class VgpStats(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("n_leaves", C.c_int64), ("n_instances", C.c_int64),
                ("n_train", C.c_int64), ("n_queries", C.c_int64), ("n_groups", C.c_int64),
                ("bucket_count", C.c_int64 * 5), ("sum_n3", C.c_double), ("sum_n2", C.c_double),
                ("t_solve_ms", C.c_double), ("t_bucket_ms", C.c_double * 5),
                ("cfg_threads", C.c_int32 * 5), ("cfg_per_sm", C.c_int32 * 5), ("grid_leaves", C.c_int64), ("grid_capacity_leaves", C.c_int64),
                ("cfg_stage_panel", C.c_int32), ("reserved", C.c_int32),
                ("graph_replays", C.c_int64), ("graph_instantiations", C.c_int64),
                ("t_bin_ms", C.c_double), ("t_gather_ms", C.c_double), ("t_fuse_ms", C.c_double),
                ("n_candidates", C.c_int64)]


# (name, restype, argtypes)
_vp, _i64, _i32 = C.c_void_p, C.c_int64, C.c_int
_PP = C.POINTER(C.c_void_p)
SIGNATURES = [
    ("vgp_default_params", None, [C.POINTER(VgpParams)]),
    ("vgp_create", _i32, [C.POINTER(VgpParams), _PP]),
    ("vgp_destroy", _i32, [_vp]),
    ("vgp_build_frame", _i32, [_vp, _vp, _i64, _vp, _vp, _PP]),
    ("vgp_frame_results", _i32, [_vp, C.POINTER(C.c_int64), _PP, _PP, _PP, _PP, _PP]),
    ("vgp_frame_instances", _i32, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _PP, _PP, _PP, _PP, _PP]),
    ("vgp_frame_destroy", _i32, [_vp]),
    ("vgp_build_frame_props", _i32, [_vp, _vp, _vp, _i64, _vp, _vp, _PP]),
    ("vgp_frame_props", _i32, [_vp, C.POINTER(C.c_int32), _PP, _PP]),
    ("vgp_export_props", _i32, [_vp, C.POINTER(C.c_int64), _vp, _vp, _vp, _vp]),
    ("vgp_import_props", _i32, [_vp, _i64, _vp, _vp, _vp, _vp]),
    ("vgp_mesh_props", _i32, [_vp, C.POINTER(C.c_int32), _PP, _PP]),
    ("vgp_fuse", _i32, [_vp, _vp, _vp]),
    ("vgp_export_grid", _i32, [_vp, C.POINTER(C.c_int64), _vp, _vp, _vp, _vp, _vp]),
    ("vgp_import_grid", _i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    ("vgp_set_surface", _i32, [_vp, _vp, _i64, _vp]),
    ("vgp_query_distance_gradient", _i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp]),
    ("vgp_query_backward", _i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp]),
    ("vgp_autotune", _i32, [_vp, _vp, _i64, _vp]),
    ("vgp_set_launch", _i32, [_vp, _vp, _vp, C.c_int32]),
    ("vgp_query_smooth", _i32, [_vp, _vp, _i64, C.c_int32, C.c_double, _vp, _vp, _vp, _vp, _vp]),
    ("vgp_extract_mesh", _i32, [_vp, _i32, _i32, _vp, _PP]),
    ("vgp_mesh_crossings", _i32, [_vp, C.POINTER(C.c_int64), _PP, _PP, _PP]),
    ("vgp_mesh_triangles", _i32, [_vp, C.POINTER(C.c_int64), _PP, _PP, _PP]),
    ("vgp_mesh_destroy", None, [_vp]),
    ("vgp_debug_mc_table", None, [_vp, _vp]),
    ("vgp_update_surface", _i32, [_vp, _vp]),
    ("vgp_surface_points", _i32, [_vp, C.POINTER(C.c_int64), _PP]),
    ("vgp_gp_batch", _i32, [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("vgp_gp_batch_static", _i32, [C.POINTER(VgpParams), _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    ("vgp_get_stats", _i32, [_vp, C.POINTER(VgpStats)]),
    ("vgp_sync", _i32, [_vp]),
    ("vgp_launch_count", C.c_int64, []),
    ("vgp_debug_exp_neg", _i32, [_vp, _vp, _vp, _i64, _vp]),
    ("vgp_debug_kernel_fix", _i32, [_vp, _vp, _vp, _i64, _vp, _vp]),
    ("vgp_debug_query_plan", _i32, [_vp, _vp, _i64, _vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _vp, _vp, _vp,
                                    _vp]),
    ("vgp_debug_smooth_plan", _i32, [_vp, _vp, _i64, C.c_int32, _vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                     _vp, _vp, _vp, _vp]),
    ("vgp_last_error", C.c_char_p, []),
]

_lib = None


class VgpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def load(path: str | None = None):
    """Load ``libvgpdf.so`` (raises if it is missing; build it with ``build.build()``)."""
    global _lib
    if _lib is None:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise ImportError(f"{p} is not built; run paper_2407_09649_gb300.build.build() "
                              "(needs nvcc) -- there is no CPU fallback")
        L = C.CDLL(p)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(rc: int) -> None:
    if rc != VGP_OK:
        raise VgpError(rc, load().vgp_last_error().decode(errors="replace"))
