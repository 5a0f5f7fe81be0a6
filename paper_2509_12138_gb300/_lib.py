"""ctypes binding of libgs (include/gs.h).  Argument marshalling only.

Loading fails loudly when the library is missing: there is no fallback
implementation anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

c_i64p = C.POINTER(C.c_int64)
c_i32p = C.POINTER(C.c_int32)
c_f32p = C.POINTER(C.c_float)


class GsCamera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("tan_fovx", C.c_float), ("tan_fovy", C.c_float), ("campos", C.c_float * 3),
                ("znear", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class GsProj(C.Structure):
    _fields_ = [("xy", C.c_void_p), ("conic_op", C.c_void_p), ("rgb", C.c_void_p), ("depth", C.c_void_p),
                ("radius", C.c_void_p), ("tiles", C.c_void_p)]


class GsGrad2d(C.Structure):
    _fields_ = [("dxy", C.c_void_p), ("dconic_op", C.c_void_p), ("drgb", C.c_void_p), ("fixed", C.c_void_p)]


class GsSchedule(C.Structure):
    _fields_ = [("tile_order", C.c_void_p), ("block_masks", C.c_void_p), ("job_base", C.c_void_p),
                ("jobs", C.c_void_p), ("checkpoints", C.c_void_p), ("chunk_last", C.c_void_p),
                ("stop_queue", C.c_void_p), ("max_jobs", C.c_int64),
                ("max_checkpoints", C.c_int64), ("chunk", C.c_int32), ("walk_whole_lists", C.c_int32)]


class GsUnits(C.Structure):
    _fields_ = [("n_units", C.c_int32), ("gauss_begin", c_i64p), ("gauss_count", c_i64p)]


class GsOwned(C.Structure):
    _fields_ = [("n_parts", C.c_int32), ("part_offsets", c_i64p), ("boxes", c_f32p), ("closed_hi", c_i32p)]


class GsDensifyCfg(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("percent_dense", C.c_float), ("min_opacity", C.c_float),
                ("max_screen", C.c_float), ("extent", C.c_float), ("step", C.c_int32), ("reset_interval", C.c_int32)]


class GsTrainBatchDesc(C.Structure):
    """gs_train_batch_desc (include/gs.h), field for field."""
    _fields_ = [("params", C.c_void_p), ("adam_m", C.c_void_p), ("adam_v", C.c_void_p), ("n_gauss", C.c_int64),
                ("sh_degree", C.c_int32), ("views_per_step", C.c_int32), ("units", C.POINTER(GsUnits)),
                ("cam_pool", C.c_void_p), ("gt_pool", C.c_void_p), ("mask_pool", C.c_void_p),
                ("train_views", C.c_void_p), ("n_views", C.c_int32), ("n_train", C.c_int32), ("width", C.c_int32),
                ("height", C.c_int32), ("lambda_ssim", C.c_float), ("bg", C.c_float * 3), ("lr_init", c_f32p),
                ("lr_final", c_f32p), ("lr_steps", C.c_int32), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("d_step", C.c_void_p), ("cams_step", C.c_void_p), ("gt_step", C.c_void_p),
                ("mask_step", C.c_void_p), ("proj", C.POINTER(GsProj)), ("max_instances", C.c_int64),
                ("sort_ws", C.c_void_p), ("sort_ws_bytes", C.c_size_t), ("sorted_vals", C.c_void_p),
                ("ranges", C.c_void_p), ("d_num_instances", C.c_void_p), ("sched", C.POINTER(GsSchedule)),
                ("img", C.c_void_p), ("final_T", C.c_void_p), ("n_contrib", C.c_void_p), ("loss_ws", C.c_void_p),
                ("loss_ws_bytes", C.c_size_t), ("d_loss", C.c_void_p), ("dL_dimg", C.c_void_p),
                ("g2d", C.POINTER(GsGrad2d)), ("grads", C.c_void_p), ("variant", C.c_int32),
                ("sparse_adam", C.c_int32),
                ("lambda_bg", C.c_float), ("bg_ws", C.c_void_p), ("bg_ws_bytes", C.c_size_t),
                ("dL_dT", C.c_void_p)]


assert C.sizeof(GsCamera) == 96

VP = C.c_void_p
I64 = C.c_int64
I32 = C.c_int
F32 = C.c_float
SZ = C.c_size_t

# name -> (restype, argtypes)
SIGNATURES = {
    "gs_param_planes": (I32, [I32]),
    "gs_status_read": (I32, [VP, I32, VP]),
    "gs_preprocess": (I32, [VP, I64, I32, C.POINTER(GsUnits), VP, I32, I32, C.POINTER(GsOwned), C.POINTER(GsProj),
                            VP, VP]),
    "gs_bin_sort_workspace_size": (SZ, [I64, I64]),
    "gs_bin_sort": (I32, [C.POINTER(GsProj), C.POINTER(GsUnits), I32, I32, I64, VP, SZ, VP, VP, VP,
                          C.POINTER(GsSchedule), VP, VP]),
    "gs_schedule_sizes": (I32, [I32, I32, I32, I64, I32, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "gs_bin_sort_static": (I32, [C.POINTER(GsProj), C.POINTER(GsUnits), I32, I32, VP, VP, VP, VP, VP]),
    "gs_bin_sort_bucketed": (I32, [C.POINTER(GsProj), C.POINTER(GsUnits), I32, I32, I64, VP, SZ, VP, VP, VP,
                                 C.POINTER(GsSchedule), VP, VP]),
    "gs_bin_sort_global": (I32, [C.POINTER(GsProj), C.POINTER(GsUnits), I32, I32, I64, VP, SZ, VP, VP, VP,
                                 C.POINTER(GsSchedule), VP, VP]),
    "gs_render_fwd": (I32, [C.POINTER(GsProj), VP, VP, I32, I32, I32, c_f32p, VP, VP, VP, I32,
                            C.POINTER(GsSchedule), VP]),
    "gs_blend_pairs": (I32, [C.POINTER(GsProj), VP, VP, I32, I32, I32, VP, VP, VP, VP]),
    "gs_loss_workspace_size": (SZ, [I32, I32, I32]),
    "gs_peak_threads": (I32, [I32]),
    "gs_peak_issue": (I32, [I32, I32, I32, F32, F32, VP, VP]),
    "gs_loss": (I32, [VP, VP, VP, I32, I32, I32, F32, VP, SZ, VP, VP, VP]),
    "gs_render_bwd": (I32, [VP, I64, I32, C.POINTER(GsUnits), VP, C.POINTER(GsProj), VP, VP, I32, I32, c_f32p, VP,
                            VP, VP, VP, VP, C.POINTER(GsGrad2d), VP, I32, C.POINTER(GsSchedule), VP]),
    "gs_blend_bwd": (I32, [C.POINTER(GsProj), VP, VP, I32, I32, I32, c_f32p, VP, VP, VP, VP, VP, C.POINTER(GsGrad2d),
                           I64, I32, C.POINTER(GsSchedule), VP]),
    "gs_bg_penalty_workspace_size": (SZ, [I32]),
    "gs_bg_penalty": (I32, [VP, VP, I32, I32, I32, F32, VP, SZ, VP, VP, VP]),
    "gs_project_bwd": (I32, [VP, I64, I32, C.POINTER(GsUnits), VP, C.POINTER(GsProj), C.POINTER(GsGrad2d), VP, VP]),
    "gs_adam_step": (I32, [VP, VP, VP, VP, I64, I32, c_f32p, c_f32p, I32, F32, F32, F32, VP, I32, VP, VP]),
    "gs_step_advance": (I32, [VP, VP]),
    "gs_project_bwd_adam": (I32, [VP, I64, I32, C.POINTER(GsUnits), VP, C.POINTER(GsProj), C.POINTER(GsGrad2d), VP,
                                  VP, c_f32p, c_f32p, I32, F32, F32, F32, VP, VP, I32, VP, VP]),
    "gs_project_bwd_adam_next": (I32, [VP, I64, I32, C.POINTER(GsUnits), VP, C.POINTER(GsProj),
                                       C.POINTER(GsGrad2d), VP, VP, c_f32p, c_f32p, I32, F32, F32, F32, VP, VP, I32,
                                       VP, I32, I32, VP, VP]),
    "gs_knn_workspace_size": (SZ, [I64, c_i32p]),
    "gs_knn": (I32, [VP, I64, I32, c_f32p, F32, c_i32p, VP, SZ, VP, VP, VP]),
    "gs_mlp_param_count": (I32, []),
    "gs_mlp_features": (I32, [VP, VP, VP, VP, I64, VP, VP]),
    "gs_mlp_forward": (I32, [VP, VP, VP, VP, I64, VP, VP, VP]),
    "gs_mlp_train_step": (I32, [VP, VP, VP, VP, VP, I64, VP, VP, VP, VP, F32, VP, VP, VP]),
    "gs_init_gaussians": (I32, [VP, VP, VP, VP, I32, I64, VP, F32, VP, I64, VP]),
    "gs_merge_render": (I32, [VP, I64, I32, C.POINTER(GsOwned), VP, I32, I32, c_f32p, C.POINTER(GsProj), I64, VP, SZ,
                              VP, VP, VP, VP, VP, VP, C.POINTER(GsSchedule), VP, VP]),
    "gs_densify_stats": (I32, [C.POINTER(GsProj), C.POINTER(GsGrad2d), C.POINTER(GsUnits), I32, I32, VP, VP, VP,
                               VP]),
    "gs_densify_workspace_size": (SZ, [I64]),
    "gs_densify_plan": (I32, [VP, I64, VP, VP, VP, C.POINTER(GsDensifyCfg), VP, SZ, VP, VP]),
    "gs_densify_apply": (I32, [VP, VP, VP, I64, I32, VP, VP, SZ, VP, VP, VP, I64, VP, VP]),
    "gs_opacity_reset": (I32, [VP, VP, VP, I64, F32, VP]),
    "gs_train_batch": (I32, [C.POINTER(GsTrainBatchDesc), VP, VP]),
    "gs_gather_views": (I32, [C.POINTER(GsTrainBatchDesc), VP, VP]),
}

OPTIONAL = set()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgs.so, building it first if needed.  Raises if it cannot be loaded."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libgs is not built ({path}); run paper_2509_12138_gb300/build.py")
        L = C.CDLL(path, mode=C.RTLD_GLOBAL)
        for name, (res, args) in SIGNATURES.items():
            if not hasattr(L, name):
                if name in OPTIONAL:
                    continue
                raise RuntimeError(f"libgs is missing symbol {name}")
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


class GsError(RuntimeError):
    pass


def check(code: int, what: str):
    if code != 0:
        raise GsError(f"{what} failed with status {code}")
