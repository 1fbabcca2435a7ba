"""ctypes declarations of include/vrc.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvrc.so")

c_i32, c_i64, c_u64, c_f32, c_f64, c_p = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float,
                                          ctypes.c_double, ctypes.c_void_p)

VRC_OK, VRC_PENDING = 0, 1
STATUS = {0: "VRC_OK", 1: "VRC_PENDING", -1: "VRC_E_INVAL", -2: "VRC_E_NOMEM", -3: "VRC_E_CUDA",
          -4: "VRC_E_TIMEOUT", -5: "VRC_E_BADID", -6: "VRC_E_BUSY", -7: "VRC_E_NONFINITE", -8: "VRC_E_INJECTED",
          -9: "VRC_E_UNSUPPORTED", -10: "VRC_E_SOURCE"}
DTYPES = {"f32": 0, "bf16": 1, "fp8": 2}
SAMPLING = {"nearest": 0, "trilinear": 1}
PATHS = {"fused": 0, "sortlast": 1, "fused_ldg": 2, "zerocopy": 3, "slab": 4}
PATH_NAMES = {0: "fused", 1: "sortlast", 2: "fused_ldg", 3: "zerocopy", 4: "slab", 5: "streamed", 6: "rows"}
COPY = {"auto": 0x000, "required": 0x100, "none": 0x200}
INJECT = {"none": 0, "alloc": 1, "h2d": 2, "drop": 3, "slab_wait": 4}


class vrc_config(ctypes.Structure):
    _fields_ = [("device", c_i32), ("n_streams", c_i32), ("max_inflight", c_i32), ("reserved0", c_i32),
                ("hbm_budget_bytes", c_i64)]


class vrc_stats(ctypes.Structure):
    _fields_ = [("min", c_f64), ("max", c_f64), ("mean", c_f64), ("std", c_f64), ("n", c_u64),
                ("n_nonfinite", c_u64)]


class vrc_camera(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("eye", c_f32 * 3), ("center", c_f32 * 3), ("up", c_f32 * 3),
                ("fovy_deg", c_f32), ("ortho_height", c_f32)]


class vrc_raycfg(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("step", c_f32), ("sampling", c_i32),
                ("opacity_correction", c_i32), ("path", c_i32), ("tile_w", c_i32), ("tile_h", c_i32),
                ("skip_empty", c_i32), ("reserved", c_i32)]


class vrc_tuning(ctypes.Structure):
    _fields_ = [("tile_w", c_i32), ("tile_h", c_i32), ("ctas_per_sm", c_i32), ("brick", c_i32), ("step", c_f32),
                ("reserved", c_i32), ("best_ms", c_f64), ("default_ms", c_f64), ("step_max_abs_diff", c_f64)]


class vrc_request(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("nbins", c_i32), ("cube_id", c_i64), ("cam", vrc_camera), ("rc", vrc_raycfg),
                ("tf_rgba", c_f32 * 1024), ("term_alpha", c_f32), ("reserved", c_i32), ("out", c_p)]


class vrc_result(ctypes.Structure):
    _fields_ = [("status", c_i32), ("path", c_i32), ("stats", vrc_stats), ("queue_ms", c_f64),
                ("latency_ms", c_f64), ("samples", c_u64), ("memory_wait_ms", c_f64), ("cube_loaded", c_i32),
                ("reserved", c_i32)]


# vrc_brick_source_fn: int32 (*)(void *user, int64 brick, int32 bx, int32 by, int32 bz, float *dst)
BRICK_SOURCE_FN = ctypes.CFUNCTYPE(c_i32, c_p, c_i64, c_i32, c_i32, c_i32, ctypes.POINTER(c_f32))

# name -> (restype, argtypes); mirrors include/vrc.h
PROTOTYPES = {
    "vrc_create": (c_i32, [ctypes.POINTER(c_p), ctypes.POINTER(vrc_config)]),
    "vrc_destroy": (c_i32, [c_p]),
    "vrc_status_str": (ctypes.c_char_p, [c_i32]),
    "vrc_last_error": (ctypes.c_char_p, [c_p]),
    "vrc_memory": (c_i32, [c_p, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    "vrc_cube_upload": (c_i32, [c_p, c_p, c_i32, c_i64, c_i64, c_i64, c_i32, c_i32, c_p, ctypes.POINTER(c_i64)]),
    "vrc_cube_register": (c_i32, [c_p, c_p, c_i64, c_i64, c_i64, c_i32, c_i32, ctypes.POINTER(c_i64)]),
    "vrc_residency": (c_i32, [c_p, ctypes.POINTER(c_i64), ctypes.POINTER(c_u64), ctypes.POINTER(c_u64)]),
    "vrc_last_render_path": (c_i32, [c_p, ctypes.POINTER(c_i32)]),
    "vrc_cube_create_streamed": (c_i32, [c_p, c_i64, c_i64, c_i64, c_i32, c_i64, c_i32, ctypes.POINTER(c_i64)]),
    "vrc_cube_put_brick": (c_i32, [c_p, c_i64, c_i64, c_p]),
    "vrc_cube_upload_streamed": (c_i32, [c_p, c_p, c_p, c_i64, c_i64, c_i64, c_i32, c_i32, c_i64, c_i32,
                                         ctypes.POINTER(c_i64)]),
    "vrc_cube_read_brick": (c_i32, [c_p, c_i64, c_i64, c_p, c_i64]),
    "vrc_cube_free": (c_i32, [c_p, c_i64]),
    "vrc_cube_free_async": (c_i32, [c_p, c_i64, c_p]),
    "vrc_cube_info": (c_i32, [c_p, c_i64, c_p, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32), ctypes.POINTER(c_i64),
                              ctypes.POINTER(c_i64), ctypes.POINTER(c_f32), ctypes.POINTER(c_f32),
                              ctypes.POINTER(c_i64)]),
    "vrc_cube_stats": (c_i32, [c_p, c_i64, c_i32, ctypes.POINTER(vrc_stats), c_p, c_p]),
    "vrc_cube_stats_async": (c_i32, [c_p, c_i64, c_i32, c_p, c_p, c_p]),
    "vrc_cube_stats_noalloc": (c_i32, [c_p, c_i64, c_i32, c_p, c_p, c_p]),
    "vrc_cube_median": (c_i32, [c_p, c_i64, ctypes.POINTER(c_f64), c_p]),
    "vrc_render_mip": (c_i32, [c_p, c_i64, ctypes.POINTER(vrc_camera), c_i32, ctypes.POINTER(vrc_raycfg), c_p, c_p]),
    "vrc_render_dvr": (c_i32, [c_p, c_i64, ctypes.POINTER(vrc_camera), c_i32, ctypes.POINTER(vrc_raycfg), c_p, c_f32,
                               c_p, c_p]),
    "vrc_last_render_samples": (c_i32, [c_p, ctypes.POINTER(c_u64), ctypes.POINTER(c_u64)]),
    "vrc_last_render_bricks": (c_i32, [c_p, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    "vrc_composite": (c_i32, [c_p, c_p, c_p, c_p, c_i64, c_i32, c_p]),
    "vrc_graph_create": (c_i32, [c_p, c_i64, ctypes.POINTER(vrc_camera), c_i32, ctypes.POINTER(vrc_raycfg), c_p,
                                 c_f32, c_p, ctypes.POINTER(c_p)]),
    "vrc_graph_launch": (c_i32, [c_p, c_p]),
    "vrc_graph_destroy": (c_i32, [c_p]),
    "vrc_autotune": (c_i32, [c_p, c_i64, ctypes.POINTER(vrc_camera), c_i32, ctypes.POINTER(vrc_raycfg), c_p, c_f32,
                             c_p, c_p, ctypes.POINTER(vrc_tuning)]),
    "vrc_autotune_cube": (c_i32, [c_p, c_i64, ctypes.POINTER(vrc_camera), c_i32, ctypes.POINTER(vrc_raycfg), c_p,
                                  c_f32, c_p, c_p, c_i32, c_f32, ctypes.POINTER(vrc_tuning)]),
    "vrc_submit": (c_i32, [c_p, ctypes.POINTER(vrc_request), ctypes.POINTER(c_u64)]),
    "vrc_poll": (c_i32, [c_p, c_u64, ctypes.POINTER(vrc_result), c_i32]),
    "vrc_debug_inject": (c_i32, [c_p, c_i32, c_i64]),
    "vrc_launch_count": (c_u64, [c_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libvrc.so.  Raises if the library has not been built: there is no
    fallback implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libvrc.so not found at {path}; build it with "
                               "`python paper_1111_6661_b300/build.py` (no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
