"""ctypes binding of the C ABI in ``include/mvtsdf.h`` (argument marshalling only).

Every ``mv_*`` function of the header is exposed here under the same name with
the same arguments; all computation happens in ``libmvtsdf.so``.  There is no
fallback: if the library is missing or cannot be loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmvtsdf.so")

MV_OK, MV_ERR_ARG, MV_ERR_OOM, MV_ERR_CUDA, MV_ERR_NOT_FOUND = 0, 1, 2, 3, 4
MV_ERR_NOT_RESIDENT, MV_ERR_BUSY, MV_ERR_DEVICE_TIMEOUT, MV_ERR_CAPACITY = 5, 6, 7, 8
STATUS_NAMES = {0: "MV_OK", 1: "MV_ERR_ARG", 2: "MV_ERR_OOM", 3: "MV_ERR_CUDA", 4: "MV_ERR_NOT_FOUND",
                5: "MV_ERR_NOT_RESIDENT", 6: "MV_ERR_BUSY", 7: "MV_ERR_DEVICE_TIMEOUT",
                8: "MV_ERR_CAPACITY"}
MV_TSDF_F32, MV_TSDF_F16, MV_TSDF_I16 = 0, 1, 2
FORMATS = {"f32": MV_TSDF_F32, "f16": MV_TSDF_F16, "i16": MV_TSDF_I16}


class mv_intrinsics(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class mv_config(C.Structure):
    _fields_ = [("trunc_voxels", C.c_float), ("w_max", C.c_float), ("color_w_max", C.c_int32),
                ("z_min", C.c_float), ("z_max", C.c_float), ("ray_step", C.c_float),
                ("n_bisect", C.c_int32)]


class mv_volume_desc(C.Structure):
    _fields_ = [("h_t", C.c_int32 * 3), ("h_r", C.c_int32 * 3), ("voxel_size", C.c_float),
                ("fmt", C.c_int32)]


class mv_volume_info(C.Structure):
    _fields_ = [("desc", mv_volume_desc), ("resident", C.c_int32), ("reserved", C.c_int32),
                ("device_bytes", C.c_uint64), ("host_bytes", C.c_uint64)]


class mv_stats(C.Structure):
    _fields_ = [("swept", C.c_uint64), ("updated", C.c_uint64), ("band", C.c_uint64),
                ("bricks", C.c_uint64), ("rays", C.c_uint64), ("ray_samples", C.c_uint64),
                ("ray_skips", C.c_uint64), ("ray_hits", C.c_uint64), ("stream_up", C.c_uint64),
                ("stream_down", C.c_uint64)]


MV_KERNEL_KINDS = 13
KERNEL_NAMES = {0: "setup", 1: "brick_list", 2: "integrate", 3: "raycast", 4: "flags",
                5: "cell_masks", 6: "backward", 7: "frame_graph", 8: "depth_tiles",
                9: "extract", 10: "depth_maps", 11: "icp",
                12: "stream"}


class mv_timings(C.Structure):
    _fields_ = [("launches", C.c_uint64 * MV_KERNEL_KINDS), ("ms", C.c_double * MV_KERNEL_KINDS),
                ("timed", C.c_uint64 * MV_KERNEL_KINDS)]


class mv_tuning(C.Structure):
    _fields_ = [("raycast_tile", C.c_int32), ("integrate_ctas_per_sm", C.c_int32),
                ("raycast_ms", C.c_float * 4), ("integrate_ms", C.c_float * 5),
                ("work_list_levels", C.c_int32)]


class mv_grad_target(C.Structure):
    _fields_ = [("id", C.c_int32), ("grad_tsdf", C.c_void_p)]


MV_NOALLOC_MAX_BRICKS = 262144


class mv_volume_view(C.Structure):
    _fields_ = [("desc", mv_volume_desc), ("fw", C.c_void_p), ("rgba", C.c_void_p),
                ("brick_flags", C.c_void_p)]


class mv_placement_config(C.Structure):
    _fields_ = [("cell_voxels", C.c_int32), ("volume_voxels", C.c_int32), ("voxel_size", C.c_float),
                ("fmt", C.c_int32), ("max_volumes", C.c_int32), ("hysteresis", C.c_float),
                ("min_count", C.c_int32)]


class mv_placement_result(C.Structure):
    _fields_ = [("cells", C.c_int32), ("added", C.c_int32), ("restored", C.c_int32),
                ("evicted", C.c_int32), ("resident", C.c_int32)]


class mv_icp_config(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("dist", C.c_float), ("cos_min", C.c_float)]


class mv_icp_system(C.Structure):
    _fields_ = [("A", C.c_double * 36), ("b", C.c_double * 6), ("error", C.c_double), ("inliers", C.c_int64)]


_P = C.c_void_p
_D16 = C.POINTER(C.c_double)
_SIGNATURES = {
    "mv_version": ([], C.c_char_p),
    "mv_config_default": ([C.POINTER(mv_config)], C.c_int),
    "mv_create": ([C.POINTER(mv_config), C.c_int32, C.POINTER(_P)], C.c_int),
    "mv_destroy": ([_P], C.c_int),
    "mv_last_error": ([_P], C.c_char_p),
    "mv_add_volume": ([_P, C.POINTER(mv_volume_desc), C.POINTER(C.c_int32)], C.c_int),
    "mv_remove_volume": ([_P, C.c_int32], C.c_int),
    "mv_query": ([_P, C.c_int32, C.POINTER(mv_volume_info)], C.c_int),
    "mv_list_volumes": ([_P, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_int32)], C.c_int),
    "mv_integrate": ([_P, _P, _P, C.POINTER(mv_intrinsics), _D16, _P], C.c_int),
    "mv_integrate_volume": ([_P, C.c_int32, _P, _P, C.POINTER(mv_intrinsics), _D16, _P], C.c_int),
    "mv_raycast": ([_P, C.POINTER(mv_intrinsics), _D16, _P, _P, _P, _P, _P, _P], C.c_int),
    "mv_raycast_batch": ([_P, C.POINTER(mv_intrinsics), _D16, C.c_int32, _P, _P, _P, _P, _P, _P], C.c_int),
    "mv_frame": ([_P, _P, _P, C.POINTER(mv_intrinsics), _D16, _P, _P, _P, _P, _P, _P], C.c_int),
    "mv_frame_host": ([_P, _P, _P, C.POINTER(mv_intrinsics), _D16, _P, _P, _P, _P, _P, C.POINTER(C.c_uint64)],
                      C.c_int),
    "mv_frame_host_wait": ([_P, C.c_uint64], C.c_int),
    "mv_frame_streamed": ([_P, _P, _P, C.POINTER(mv_intrinsics), _D16, _P, _P, _P, _P, _P, C.c_int32, _P],
                          C.c_int),
    "mv_raycast_volume": ([_P, C.c_int32, C.c_int32, C.POINTER(mv_intrinsics), _D16, _P, _P, _P,
                           _P, _P, _P], C.c_int),
    "mv_autotune": ([_P, _P, _P, C.POINTER(mv_intrinsics), _D16, C.POINTER(mv_tuning), _P], C.c_int),
    "mv_set_tuning": ([_P, C.POINTER(mv_tuning)], C.c_int),
    "mv_get_tuning": ([_P, C.POINTER(mv_tuning)], C.c_int),
    "mv_raycast_backward": ([_P, C.POINTER(mv_intrinsics), _D16, C.c_int32, _P, _P, _P, _P, _P,
                             C.POINTER(mv_grad_target), C.c_int32, _P], C.c_int),
    "mv_raycast_backward_l1": ([_P, C.POINTER(mv_intrinsics), _D16, C.c_int32, _P, _P, _P, _P, _P, C.c_float,
                                _P, _P, _P], C.c_int),
    "mv_swap_out": ([_P, C.c_int32, _P], C.c_int),
    "mv_swap_in": ([_P, C.c_int32, _P], C.c_int),
    "mv_read_volume": ([_P, C.c_int32, _P, _P], C.c_int),
    "mv_read_box": ([_P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32), _P, _P], C.c_int),
    "mv_write_volume": ([_P, C.c_int32, _P, _P], C.c_int),
    "mv_read_brick_flags": ([_P, C.c_int32, _P, C.c_uint64], C.c_int),
    "mv_get_stats": ([_P, C.POINTER(mv_stats), C.c_int32], C.c_int),
    "mv_set_timing": ([_P, C.c_int32], C.c_int),
    "mv_get_timings": ([_P, C.POINTER(mv_timings), C.c_int32], C.c_int),
    "mv_synchronize": ([_P], C.c_int),
    "mv_integrate_noalloc": ([C.POINTER(mv_volume_view), C.POINTER(mv_config), _P, _P,
                              C.POINTER(mv_intrinsics), _D16, _P], C.c_int),
    "mv_pack_hits": ([_P, _P, _P, C.c_int32, C.c_int64, _P, _P], C.c_int),
    "mv_merge_hits": ([_P, _P, C.c_int64, _P, _P, _P, _P, _P, _P], C.c_int),
    "mv_get_config": ([_P, C.POINTER(mv_config)], C.c_int),
    "mv_reserve_host": ([_P, C.POINTER(mv_volume_desc), C.c_int32], C.c_int),
    "mv_depth_to_maps": ([_P, _P, C.POINTER(mv_intrinsics), _D16, _P, _P, _P], C.c_int),
    "mv_icp_linearize": ([_P, _P, _P, C.POINTER(mv_intrinsics), _D16, _P, _P, _D16, C.POINTER(mv_icp_config),
                       C.POINTER(mv_icp_system), _P], C.c_int),
    "mv_track": ([_P, _P, C.POINTER(mv_intrinsics), _P, _P, _D16, _D16, C.POINTER(mv_icp_config), _D16,
                  C.POINTER(mv_icp_system), _P], C.c_int),
    "mv_extract_points": ([_P, C.c_int32, _P, _P, _P, C.c_uint64, C.POINTER(C.c_uint64), _P], C.c_int),
    "mv_get_device": ([_P], C.c_int32),
    "mv_placer_create": ([_P, C.POINTER(mv_placement_config), C.POINTER(_P)], C.c_int),
    "mv_placer_destroy": ([_P], C.c_int),
    "mv_placer_last_error": ([_P], C.c_char_p),
    "mv_placer_histogram": ([_P, _P, C.POINTER(mv_intrinsics), _D16, C.POINTER(C.c_int32),
                             C.POINTER(C.c_uint32), C.c_int32, C.POINTER(C.c_int32), _P], C.c_int),
    "mv_placer_update": ([_P, _P, C.POINTER(mv_intrinsics), _D16, C.POINTER(mv_placement_result), _P],
                         C.c_int),
    "mv_placer_list": ([_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int32,
                        C.POINTER(C.c_int32)], C.c_int),
}

_lib = None


def lib() -> C.CDLL:
    """Load libmvtsdf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1511_07106_b300.build` (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def declared_functions():
    return list(_SIGNATURES)


class MVError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def __getattr__(name):
    # mv_* names resolve to the C functions themselves
    if name in _SIGNATURES:
        return getattr(lib(), name)
    raise AttributeError(name)
