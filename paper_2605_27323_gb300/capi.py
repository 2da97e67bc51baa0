"""ctypes declarations of include/pt.h and the loader of the in-tree libpt.so.

Argument marshalling only: every step of rendering runs in the library's CUDA kernels.  There is no
CPU fallback; if the library is missing this module raises instead of degrading.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

u32, u64, f32, vp = C.c_uint32, C.c_uint64, C.c_float, C.c_void_p

PT_OK = 0
STATUS_NAMES = {0: "PT_OK", 1: "PT_ERR_INVALID_ARG", 2: "PT_ERR_OOM", 3: "PT_ERR_CUDA",
                4: "PT_ERR_QUEUE_OVERFLOW", 5: "PT_ERR_TRAVERSAL_LIMIT", 6: "PT_ERR_TIMEOUT",
                7: "PT_ERR_UNSUPPORTED"}
MODE = {"megakernel": 0, "wavefront": 1}
SORT = {"none": 0, "type": 1, "material": 2}
FLAG_PROFILE, FLAG_NO_GRAPH, FLAG_MK_STATIC, FLAG_HALTON, FLAG_MIS, FLAG_SHORT_STACK, FLAG_COUNT_TRAVERSAL = (
    1, 2, 4, 8, 16, 32, 64)
FLAG_SEPARATE_SHADOW = 128

# Every function that include/pt.h declares (the symbol-export test checks this list against the
# header and the shared object).
EXPORTED = ["pt_scene_create", "pt_scene_create_instanced", "pt_scene_set_materials", "pt_render", "pt_render_progressive", "pt_render_backward",
            "pt_render_batch",
            "pt_autotune_batch", "pt_trace_closest", "pt_get_stats", "pt_debug_rng", "pt_debug_trace_paths",
            "pt_scene_info", "pt_render_wavefront_static",
            "pt_status_string", "pt_last_error", "pt_scene_destroy"]


class Material(C.Structure):
    _fields_ = [("type", u32), ("albedo", f32 * 3), ("emission", f32), ("roughness", f32), ("ior", f32),
                ("flags", u32)]


class Instance(C.Structure):
    _fields_ = [("xform", f32 * 12), ("mesh", u32), ("material", u32), ("reserved", u32 * 2)]


NO_MATERIAL = 0xFFFFFFFF


class Camera(C.Structure):
    _fields_ = [("eye", f32 * 3), ("target", f32 * 3), ("up", f32 * 3), ("vfov_deg", f32), ("width", u32),
                ("height", u32)]


class RenderOpts(C.Structure):
    _fields_ = [("mode", u32), ("rr_start", u32), ("rr_fixed", f32), ("sort_mode", u32), ("block_size", u32),
                ("flags", u32), ("queue_capacity", u64), ("d_path_sig", vp), ("hybrid_threshold", u64)]


class Stats(C.Structure):
    _fields_ = [("extension_rays", u64), ("shadow_rays", u64), ("paths", u64), ("bounces", u32), ("status", u32),
                ("active", u64 * 64), ("ms_raygen", f32), ("ms_extend", f32), ("ms_sort", f32), ("ms_shade", f32),
                ("ms_shadow", f32), ("ms_reduce", f32), ("ms_megakernel", f32), ("ms_adjoint", f32),
                ("launches_extend", u32), ("launches_shadow", u32), ("launches_total", u32), ("ms_total", f32),
                ("nodes_closest", u64), ("tris_closest", u64), ("nodes_any", u64), ("tris_any", u64),
                ("shadow_queued", u64 * 64), ("group_walks", u64 * 5)]


class PtError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpt.so (building it first when sources changed).  Raises if it cannot be built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libpt.so not found at {path}; run __graft_entry__.build()")
    L = C.CDLL(path)
    P = C.POINTER
    L.pt_scene_create.restype = u32
    L.pt_scene_create.argtypes = [vp, u32, vp, u32, vp, vp, u32, vp, vp, P(vp)]
    L.pt_scene_create_instanced.restype = u32
    L.pt_scene_create_instanced.argtypes = [u32, P(vp), P(u32), P(vp), P(u32), P(vp), P(Instance), u32, vp, u32, vp,
                                            vp, P(vp)]
    L.pt_scene_set_materials.restype = u32
    L.pt_scene_set_materials.argtypes = [vp, vp, vp, vp]
    L.pt_render.restype = u32
    L.pt_render.argtypes = [vp, P(Camera), u32, u32, u64, P(RenderOpts), vp, vp, vp]
    L.pt_render_progressive.restype = u32
    L.pt_render_progressive.argtypes = [vp, P(Camera), u32, u32, u64, u32, P(RenderOpts), vp, vp, vp]
    L.pt_render_backward.restype = u32
    L.pt_render_backward.argtypes = [vp, P(Camera), u32, u32, u64, P(RenderOpts), vp, vp, vp, vp]
    L.pt_render_batch.restype = u32
    L.pt_render_batch.argtypes = [P(vp), P(Camera), P(u32), u32, u32, u64, P(RenderOpts), P(vp), vp]
    L.pt_autotune_batch.restype = u32
    L.pt_autotune_batch.argtypes = [P(vp), P(Camera), P(u32), u32, u32, u64, P(RenderOpts), P(vp), vp,
                                    P(RenderOpts), P(f32)]
    L.pt_trace_closest.restype = u32
    L.pt_trace_closest.argtypes = [vp, vp, u32, vp, vp, vp]
    L.pt_get_stats.restype = u32
    L.pt_get_stats.argtypes = [vp, P(Stats)]
    L.pt_debug_rng.restype = u32
    L.pt_debug_rng.argtypes = [u64, vp, vp, vp, vp, u32, vp, vp]
    L.pt_debug_trace_paths.restype = u32
    L.pt_debug_trace_paths.argtypes = [vp, P(Camera), u32, u32, u64, P(RenderOpts), vp, u32, vp, vp, vp, vp, vp]
    L.pt_render_wavefront_static.restype = u32
    L.pt_render_wavefront_static.argtypes = [vp, P(Camera), u32, u32, u64, P(RenderOpts), vp, vp]
    L.pt_scene_info.restype = u32
    L.pt_scene_info.argtypes = [vp, P(u64), P(u64), P(u64), P(f32), P(u64)]
    L.pt_status_string.restype = C.c_char_p
    L.pt_status_string.argtypes = [u32]
    L.pt_last_error.restype = C.c_char_p
    L.pt_last_error.argtypes = []
    L.pt_scene_destroy.restype = None
    L.pt_scene_destroy.argtypes = [vp]
    _lib = L
    return L


def check(status: int):
    if status != PT_OK:
        msg = _lib.pt_last_error().decode(errors="replace") if _lib is not None else ""
        raise PtError(int(status), msg)
