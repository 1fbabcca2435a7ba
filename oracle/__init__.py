"""CPU oracle of the cube statistics and ray-casting path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  The product library never links,
imports or calls it, and it shares no code with the CUDA path.

The numerical definitions live in ``oracle.c`` (plain C, binary64 accumulation,
binary32 ray set-up and bin formula, compiled without FMA contraction); this
file only marshals numpy arrays.  Paper passages: min/max and histogram
(Abstract), standard deviation and median (Sec. 3), sub-cube ray casting and
gathering of partial images (Sec. 2, Table 1).

Parity status: every function here is pinned by tests/test_oracle_*.py against
closed forms, brute force or library routines independent of this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

DTYPES = {"f32": 0, "bf16": 1, "fp8": 2}


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Camera(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("eye", ctypes.c_float * 3), ("center", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("fovy_deg", ctypes.c_float), ("ortho_height", ctypes.c_float)]


class _RayCfg(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("step", ctypes.c_float),
                ("sampling", ctypes.c_int32), ("mode", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, f32 = ctypes.c_int64, ctypes.c_int32, ctypes.c_float
            lib.orc_stats.argtypes = [P, i64, P, P]
            lib.orc_histogram.argtypes = [P, i64, f32, f32, i32, P]
            lib.orc_median.argtypes = [P, i64, P]
            lib.orc_bf16_round_n.argtypes = [P, i64, P]
            lib.orc_bf16_round_n.restype = None
            lib.orc_e4m3_round_n.argtypes = [P, i64, P]
            lib.orc_e4m3_round_n.restype = None
            lib.orc_brick_scales.argtypes = [P, P, i32, P]
            lib.orc_dequantize.argtypes = [P, P, i32, i32, P, P]
            lib.orc_camera_basis.argtypes = [ctypes.POINTER(_Camera), i32, i32, P]
            lib.orc_camera_basis.restype = None
            lib.orc_ray.argtypes = [P, i32, i32, i32, P, P, P, P]
            lib.orc_render.argtypes = [P, P, i32, i32, P, ctypes.POINTER(_Camera), ctypes.POINTER(_RayCfg),
                                       P, f32, f32, f32, i32, P, i64, P, P, P, P, P]
            lib.orc_composite.argtypes = [P, P, i64, i32, P]
            lib.orc_composite.restype = None
            _lib = lib
    return _lib


def _f32(v):
    return np.ascontiguousarray(v, dtype=np.float32)


def _dims(v):
    sz, sy, sx = v.shape
    return np.array([sx, sy, sz], dtype=np.int64)


def stats(v) -> dict:
    v = _f32(v).ravel()
    out = np.zeros(4)
    cnt = np.zeros(2, dtype=np.int64)
    _load().orc_stats(v.ctypes.data, v.size, out.ctypes.data, cnt.ctypes.data)
    return dict(min=out[0], max=out[1], mean=out[2], std=out[3], n=int(cnt[0]), n_nonfinite=int(cnt[1]))


def histogram(v, vmin: float, vmax: float, nbins: int) -> np.ndarray:
    v = _f32(v).ravel()
    h = np.zeros(nbins, dtype=np.uint64)
    if _load().orc_histogram(v.ctypes.data, v.size, np.float32(vmin), np.float32(vmax), nbins, h.ctypes.data):
        raise ValueError("nbins must be positive")
    return h


def median(v) -> float:
    v = _f32(v).ravel()
    out = np.zeros(1)
    rc = _load().orc_median(v.ctypes.data, v.size, out.ctypes.data)
    if rc == -2:
        raise MemoryError
    return float(out[0])


def bf16_round(x) -> np.ndarray:
    x = _f32(x)
    out = np.empty_like(x)
    _load().orc_bf16_round_n(x.ctypes.data, x.size, out.ctypes.data)
    return out


def e4m3_round(x) -> np.ndarray:
    x = _f32(x)
    out = np.empty(x.shape, dtype=np.float64)
    _load().orc_e4m3_round_n(x.ctypes.data, x.size, out.ctypes.data)
    return out


def brick_scales(v, B: int) -> np.ndarray:
    v = _f32(v)
    d = _dims(v)
    nb = [(int(x) + B - 1) // B for x in d]
    s = np.empty(nb[0] * nb[1] * nb[2], dtype=np.float32)
    _load().orc_brick_scales(v.ctypes.data, d.ctypes.data, B, s.ctypes.data)
    return s


def dequantize(v, dtype: str, B: int = 0, scales=None) -> np.ndarray:
    """The cube as stored: every voxel rounded by the brick that owns it."""
    v = _f32(v)
    d = _dims(v)
    if dtype == "fp8" and scales is None:
        scales = brick_scales(v, B)
    sc = _f32(scales) if scales is not None else np.ones(1, np.float32)
    out = np.empty_like(v)
    _load().orc_dequantize(v.ctypes.data, d.ctypes.data, DTYPES[dtype], B, sc.ctypes.data, out.ctypes.data)
    return out


def _cam(c: dict) -> _Camera:
    cam = _Camera()
    cam.kind = int(c["kind"])
    for a in range(3):
        cam.eye[a] = c["eye"][a]
        cam.center[a] = c["center"][a]
        cam.up[a] = c["up"][a]
    cam.fovy_deg = c.get("fovy_deg", 30.0)
    cam.ortho_height = c.get("ortho_height", 1.0)
    return cam


def camera_basis(cam: dict, W: int, H: int) -> np.ndarray:
    b = np.empty(12, dtype=np.float32)
    c = _cam(cam)
    _load().orc_camera_basis(ctypes.byref(c), W, H, b.ctypes.data)
    return b


def ray(cam: dict, W: int, H: int, px: int, py: int, dims):
    """(hit, origin, direction, (t_entry, t_exit)) of one pixel, binary32."""
    b = camera_basis(cam, W, H)
    d = np.array(dims, dtype=np.int64)
    o = np.empty(3, np.float32)
    di = np.empty(3, np.float32)
    t = np.empty(2, np.float32)
    hit = _load().orc_ray(b.ctypes.data, int(cam["kind"]), px, py, d.ctypes.data, o.ctypes.data,
                          di.ctypes.data, t.ctypes.data)
    return bool(hit), o, di, t


def render(v, cam: dict, W: int, H: int, step: float, sampling: str = "trilinear", mode: str = "mip",
           tf=None, vmin: float = 0.0, vmax: float = 1.0, term: float = 0.99, opacity_correction: bool = False,
           pixels=None, dtype: str = "f32", brick: int = 0, scales=None) -> dict:
    """Render the given pixels (flat indices py*W+px; default all) of one view.

    Returns dict(out, lo, hi, fragile, nsamp).  MIP: out has one value per
    pixel.  DVR: out/lo/hi have 4 per pixel (premultiplied RGBA).
    """
    v = _f32(v)
    d = _dims(v)
    if pixels is None:
        pixels = np.arange(W * H, dtype=np.int64)
    pixels = np.ascontiguousarray(pixels, dtype=np.int64)
    n = pixels.size
    m = 0 if mode == "mip" else 1
    if dtype == "fp8":
        if brick <= 0:
            raise ValueError("fp8 storage is defined per brick")
        if scales is None:
            scales = brick_scales(v, brick)
    sc = _f32(scales) if scales is not None else np.ones(1, np.float32)
    tf_arr = _f32(tf if tf is not None else np.zeros((256, 4)))
    out = np.empty(n * (1 if m == 0 else 4))
    lo = np.empty(n * 4) if m else None
    hi = np.empty(n * 4) if m else None
    flags = np.zeros(n, dtype=np.int32)
    nsamp = np.zeros(n, dtype=np.int64)
    rc = _RayCfg(W, H, step, {"nearest": 0, "trilinear": 1}[sampling], m)
    c = _cam(cam)
    r = _load().orc_render(v.ctypes.data, d.ctypes.data, DTYPES[dtype], brick, sc.ctypes.data,
                           ctypes.byref(c), ctypes.byref(rc), tf_arr.ctypes.data, np.float32(vmin),
                           np.float32(vmax), np.float32(term), int(opacity_correction), pixels.ctypes.data, n,
                           out.ctypes.data, lo.ctypes.data if m else None, hi.ctypes.data if m else None,
                           flags.ctypes.data, nsamp.ctypes.data)
    if r == -3:
        raise AssertionError("brick visibility order disagrees with ray order")
    if m:
        out, lo, hi = out.reshape(n, 4), lo.reshape(n, 4), hi.reshape(n, 4)
    return dict(out=out, lo=lo, hi=hi, fragile=flags.astype(bool), nsamp=nsamp)


def composite(front, back, mode: str = "dvr") -> np.ndarray:
    f = np.ascontiguousarray(front, dtype=np.float64)
    b = np.ascontiguousarray(back, dtype=np.float64)
    out = np.empty_like(f)
    npix = f.size if mode == "mip" else f.size // 4
    _load().orc_composite(f.ctypes.data, b.ctypes.data, npix, 0 if mode == "mip" else 1, out.ctypes.data)
    return out
