"""ctypes mirror of include/vct.h and the loader of libvct.so."""
from __future__ import annotations

import contextlib
import ctypes
import os
import threading

from . import build as _build

MAX_DIFFUSE = 32
MAX_PYRAMIDS = 8
MAX_LEVELS = 11

VCT_OK, VCT_ERR_INVALID_ARG, VCT_ERR_CUDA, VCT_ERR_WORKSPACE, VCT_ERR_UNSUPPORTED, \
    VCT_ERR_TIMEOUT = range(6)
VCT_F32, VCT_F16 = 0, 1
LAYOUT_DENSE, LAYOUT_BRICKS, LAYOUT_ANISO = 0, 1, 2
FLAG_OCC_SMOOTH, FLAG_SPEC_GRACE, FLAG_DIFFUSE_FIRST_HIT, FLAG_SHADE, FLAG_SHADE_IMPL, \
    FLAG_PREMULTIPLIED = 1, 2, 4, 8, 16, 32

_c_i32, _c_u64, _c_f32, _vp = ctypes.c_int32, ctypes.c_uint64, ctypes.c_float, ctypes.c_void_p


class VctPyramid(ctypes.Structure):
    _fields_ = [("n", _c_i32), ("levels", _c_i32), ("dtype", _c_i32), ("layout", _c_i32),
                ("origin", _c_f32 * 3), ("size", _c_f32), ("data", _vp), ("bytes", _c_u64)]


class VctTraceParams(ctypes.Structure):
    _fields_ = [("n_diffuse", _c_i32), ("spec_enable", _c_i32), ("occ_enable", _c_i32),
                ("flags", _c_i32),
                ("diffuse_dir", (_c_f32 * 3) * MAX_DIFFUSE),
                ("diffuse_weight", _c_f32 * MAX_DIFFUSE),
                ("diffuse_aperture", _c_f32),
                ("spec_aperture_min", _c_f32), ("spec_aperture_max", _c_f32),
                ("roughness_min", _c_f32), ("occ_aperture", _c_f32),
                ("light_dir", _c_f32 * 3), ("beta", _c_f32), ("t0_voxels", _c_f32),
                ("normal_offset_voxels", _c_f32), ("t_max", _c_f32),
                ("shadow_str", _c_f32), ("occ_max_dist", _c_f32), ("shininess", _c_f32),
                ("shininess_falloff", _c_f32), ("diffuse_str", _c_f32),
                ("specular_str", _c_f32), ("light_color", _c_f32 * 3)]


class VctView(ctypes.Structure):
    _fields_ = [("width", _c_i32), ("height", _c_i32), ("pyramid", _c_i32), ("reserved", _c_i32),
                ("position", _vp), ("normal", _vp), ("roughness", _vp), ("mask", _vp),
                ("camera", _c_f32 * 3), ("pad", _c_f32),
                ("out_diffuse", _vp), ("out_specular", _vp), ("out_visibility", _vp),
                ("albedo", _vp), ("out_radiance", _vp), ("cone_state", _vp)]


class VctLaunchConfig(ctypes.Structure):
    _fields_ = [("tile_w", _c_i32), ("tile_h", _c_i32), ("lanes_per_pixel", _c_i32),
                ("ctas_per_sm", _c_i32)]


class VctTraceStats(ctypes.Structure):
    _fields_ = [("samples", ctypes.c_uint64 * 3), ("cones", ctypes.c_uint64 * 3),
                ("queue", ctypes.c_uint32), ("status", ctypes.c_uint32)]


class VctViewGrad(ctypes.Structure):
    _fields_ = [("grad_diffuse", _vp), ("grad_specular", _vp), ("grad_visibility", _vp),
                ("grad_radiance", _vp)]


class VctMesh(ctypes.Structure):
    _fields_ = [("vertices", _vp), ("indices", _vp), ("colors", _vp), ("n_vertices", _c_i32),
                ("n_triangles", _c_i32)]


class VctVoxelLight(ctypes.Structure):
    _fields_ = [("light_dir", _c_f32 * 3), ("light_color", _c_f32 * 3), ("ambient", _c_f32),
                ("diffuse_str", _c_f32)]


class VctVoxelizeStats(ctypes.Structure):
    _fields_ = [("fragments", ctypes.c_uint64), ("large_items", ctypes.c_uint64),
                ("item_cursor", ctypes.c_uint64), ("skipped", ctypes.c_uint32),
                ("degenerate", ctypes.c_uint32), ("large_triangles", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class VctCamera(ctypes.Structure):
    _fields_ = [("eye", _c_f32 * 3), ("forward", _c_f32 * 3), ("right", _c_f32 * 3),
                ("up", _c_f32 * 3), ("tan_half_fov", _c_f32), ("width", _c_i32),
                ("height", _c_i32), ("frame_origin", _c_f32 * 3), ("frame_size", _c_f32)]


class VctGbufferStats(ctypes.Structure):
    _fields_ = [("pairs", ctypes.c_uint64), ("pair_capacity", ctypes.c_uint64),
                ("skipped", ctypes.c_uint32), ("degenerate", ctypes.c_uint32),
                ("culled", ctypes.c_uint32), ("wide", ctypes.c_uint32),
                ("overflow", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 3)]


class VctPipelineDesc(ctypes.Structure):
    _fields_ = [("n", _c_i32), ("levels", _c_i32), ("dtype", _c_i32), ("width", _c_i32),
                ("height", _c_i32), ("has_roughness", _c_i32), ("has_mask", _c_i32),
                ("outputs", _c_i32), ("origin", _c_f32 * 3), ("size", _c_f32)]


class VctHostFrame(ctypes.Structure):
    _fields_ = [("level0", _vp), ("position", _vp), ("normal", _vp), ("roughness", _vp),
                ("mask", _vp), ("camera", _c_f32 * 3), ("pad", _c_f32), ("out_diffuse", _vp),
                ("out_specular", _vp), ("out_visibility", _vp)]


EXPORTS = {
    "vct_pyramid_bytes": (ctypes.c_size_t, [_c_i32, _c_i32, _c_i32]),
    "vct_pyramid_level_offset": (_c_u64, [_c_i32, _c_i32, _c_i32, _c_i32]),
    "vct_pyramid_bytes_bricks": (ctypes.c_size_t, [_c_i32, _c_i32, _c_i32, _c_u64]),
    "vct_pyramid_bytes_aniso": (ctypes.c_size_t, [_c_i32, _c_i32, _c_i32]),
    "vct_pyramid_read_volume": (_c_i32, [ctypes.POINTER(VctPyramid), _c_i32, _c_i32, _vp, _vp]),
    "vct_pyramid_plan_scratch_bytes": (ctypes.c_size_t, [_c_i32, _c_i32, _c_i32]),
    "vct_pyramid_plan_bricks": (_c_i32, [_vp, _c_i32, _c_i32, _c_i32, _vp, ctypes.c_size_t,
                                         ctypes.POINTER(_c_u64), ctypes.POINTER(_c_u64), _vp]),
    "vct_build_mips": (_c_i32, [_vp, ctypes.POINTER(VctPyramid), _vp]),
    "vct_pyramid_read_level": (_c_i32, [ctypes.POINTER(VctPyramid), _c_i32, _vp, _vp]),
    "vct_pyramid_status": (_c_i32, [ctypes.POINTER(VctPyramid), _vp]),
    "vct_trace_workspace_bytes": (ctypes.c_size_t, []),
    "vct_trace": (_c_i32, [ctypes.POINTER(VctPyramid), _c_i32, ctypes.POINTER(VctView), _c_i32,
                           ctypes.POINTER(VctTraceParams), ctypes.POINTER(VctLaunchConfig), _vp,
                           ctypes.c_size_t, _vp]),
    "vct_autotune_trace": (_c_i32, [ctypes.POINTER(VctPyramid), _c_i32, ctypes.POINTER(VctView),
                                    _c_i32, ctypes.POINTER(VctTraceParams), _vp, ctypes.c_size_t,
                                    _vp, ctypes.POINTER(VctLaunchConfig)]),
    "vct_trace_backward_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(VctPyramid)]),
    "vct_trace_backward": (_c_i32, [ctypes.POINTER(VctPyramid), ctypes.POINTER(VctView),
                                    ctypes.POINTER(VctViewGrad), _c_i32,
                                    ctypes.POINTER(VctTraceParams),
                                    ctypes.POINTER(VctLaunchConfig), _vp, _vp, ctypes.c_size_t,
                                    _vp]),
    "vct_trace_backward_deterministic_workspace_bytes": (ctypes.c_size_t,
                                                         [ctypes.POINTER(VctPyramid)]),
    "vct_trace_backward_deterministic": (_c_i32, [ctypes.POINTER(VctPyramid),
                                                  ctypes.POINTER(VctView),
                                                  ctypes.POINTER(VctViewGrad), _c_i32,
                                                  ctypes.POINTER(VctTraceParams),
                                                  ctypes.POINTER(VctLaunchConfig), _vp, _vp,
                                                  ctypes.c_size_t, _vp]),
    "vct_trace_backward_noalloc": (_c_i32, [ctypes.POINTER(VctPyramid), ctypes.POINTER(VctView),
                                            ctypes.POINTER(VctViewGrad), _c_i32,
                                            ctypes.POINTER(VctTraceParams),
                                            ctypes.POINTER(VctLaunchConfig), _vp, _vp]),
    "vct_voxelize_workspace_bytes": (ctypes.c_size_t, [_c_i32, _c_i32]),
    "vct_voxelize": (_c_i32, [ctypes.POINTER(VctMesh), _c_i32, ctypes.POINTER(_c_f32), _c_f32,
                              ctypes.POINTER(VctVoxelLight), _vp, _vp, ctypes.c_size_t, _vp]),
    "vct_gbuffer_workspace_bytes": (ctypes.c_size_t, [_c_i32, _c_i32, _c_i32, _c_u64]),
    "vct_gbuffer": (_c_i32, [ctypes.POINTER(VctMesh), ctypes.POINTER(VctCamera), _vp, _vp, _vp,
                             _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "vct_pipeline_create": (_c_i32, [ctypes.POINTER(VctPipelineDesc),
                                     ctypes.POINTER(VctTraceParams), ctypes.POINTER(_vp)]),
    "vct_pipeline_submit": (_c_i32, [_vp, ctypes.POINTER(VctHostFrame), _vp]),
    "vct_pipeline_join": (_c_i32, [_vp, _vp]),
    "vct_pipeline_stats": (_c_i32, [_vp, _c_i32, ctypes.POINTER(VctTraceStats)]),
    "vct_pipeline_destroy": (None, [_vp]),
    "vct_status_string": (ctypes.c_char_p, [_c_i32]),
    "vct_last_error": (ctypes.c_char_p, []),
    "vct_version": (_c_i32, []),
    "vct_debug_wait_probe": (_c_i32, [_vp, _c_u64, _vp]),
    "vct_debug_bounds_flags": (_c_i32, [ctypes.POINTER(ctypes.c_uint32), _c_i32]),
    "vct_debug_bounds_probe": (_c_i32, [_vp, ctypes.c_uint32, ctypes.c_uint32, _vp]),
}

_LOCK = threading.Lock()
_LIB = None


class VctError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def library_path(variant: str = "release") -> str:
    return _build.library_file(variant)


def open_library(variant: str = "release", build_if_missing: bool = True):
    """Load one variant of the library (building it first if needed) with
    its exports declared.  Raises if unavailable: there is no fallback."""
    path = _build.build(variant=variant) if build_if_missing else library_path(variant)
    if not os.path.exists(path):
        raise RuntimeError(f"{os.path.basename(path)} not found at {path}; run the build first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(build_if_missing: bool = True):
    """The library the binding calls: the release libvct.so unless
    using_variant() selected another."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = open_library("release", build_if_missing)
        return _LIB


@contextlib.contextmanager
def using_variant(variant: str):
    """Route the binding's calls to another variant of the library (e.g.
    the bounds-checked build) inside the block."""
    global _LIB
    lib = open_library(variant)
    with _LOCK:
        prev = _LIB
        _LIB = lib
    try:
        yield lib
    finally:
        with _LOCK:
            _LIB = prev


def check(status: int, what: str) -> None:
    if status != VCT_OK:
        lib = load()
        raise VctError(status, f"{what}: {lib.vct_status_string(status).decode()}: "
                               f"{lib.vct_last_error().decode()}")
