"""Seeded synthetic inputs: spectral cubes, cameras, transfer functions, request streams.

This module produces inputs only.  It contains none of the arithmetic of the
method under test (statistics, ray setup, sampling, compositing), so both the
CPU oracle and the CUDA library can be fed from it without sharing code.

The paper's case study (Sec. 2, Table 1; Sec. 3) renders real spectral data
cubes of 4-204 GB; those are not available, so cubes are generated from a seed
as N(0,1) noise plus anisotropic Gaussian sources (see ``cubegen.c``).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cubegen.c")
_LIB = os.path.join(_HERE, "libcubegen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile libcubegen.so next to its source (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32
            lib.cg_generate_box.argtypes = [i64, i64, i64, u64, i32, i64, i64, i64, i64, i64, i64,
                                            ctypes.c_void_p]
            lib.cg_generate_box.restype = ctypes.c_int
            lib.cg_sources.argtypes = [i64, i64, i64, u64, i32, ctypes.c_void_p]
            lib.cg_sources.restype = None
            lib.cg_noise.argtypes = [u64, u64]
            lib.cg_noise.restype = ctypes.c_double
            lib.cg_brick_source.argtypes = [ctypes.c_void_p, i64, i32, i32, i32, ctypes.c_void_p]
            lib.cg_brick_source.restype = i32
            _lib = lib
    return _lib


def generate(dims, n_sources: int, seed: int, box=None, out: np.ndarray | None = None) -> np.ndarray:
    """Cube (or sub-box) as float32 array of shape (sz, sy, sx), x fastest.

    dims = (nx, ny, nz); box = (x0, y0, z0, sx, sy, sz) or None for the whole cube.
    """
    nx, ny, nz = (int(d) for d in dims)
    if box is None:
        box = (0, 0, 0, nx, ny, nz)
    x0, y0, z0, sx, sy, sz = (int(b) for b in box)
    if out is None:
        out = np.empty((sz, sy, sx), dtype=np.float32)
    assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == sx * sy * sz
    rc = _load().cg_generate_box(nx, ny, nz, seed, n_sources, x0, y0, z0, sx, sy, sz,
                                 out.ctypes.data)
    if rc != 0:
        raise ValueError(f"cubegen: bad box {box} for dims {dims} or out of memory")
    return out


def sources(dims, n_sources: int, seed: int) -> np.ndarray:
    """Source table (n, 7): cx, cy, cz, peak A, sigma_x, sigma_y, sigma_z."""
    nx, ny, nz = (int(d) for d in dims)
    out = np.empty((n_sources, 7), dtype=np.float64)
    if n_sources:
        _load().cg_sources(nx, ny, nz, seed, n_sources, out.ctypes.data)
    return out


def noise(seed: int, idx: int) -> float:
    return _load().cg_noise(seed, idx)


# --------------------------------------------------------------------------- cameras
def camera(kind: str, eye, center, up, fovy_deg: float = 30.0, ortho_height: float = 1.0) -> dict:
    """Plain camera record: fields mirror ``vrc_camera`` (fp32 when marshalled)."""
    return {"kind": {"ortho": 0, "persp": 1}[kind], "eye": [float(v) for v in eye],
            "center": [float(v) for v in center], "up": [float(v) for v in up],
            "fovy_deg": float(fovy_deg), "ortho_height": float(ortho_height)}


def ortho_z_camera(dims) -> dict:
    """Orthographic view along +z covering the x-y face of the cube exactly.

    With the library's basis formula and an image of W x H pixels, pixel (u, v)
    casts its ray from (x, y) = ((u+0.5) nx/W, (v+0.5) ny/H) along +z; image
    rows grow with +y.  Requires W/H == nx/ny.
    """
    nx, ny, nz = dims
    return camera("ortho", (nx / 2, ny / 2, 0.0), (nx / 2, ny / 2, 1.0), (0.0, -1.0, 0.0),
                  ortho_height=float(ny))


def orbit_cameras(dims, n_views: int, elevation_deg: float = 20.0, dist_factor: float = 1.5,
                  fovy_deg: float = 30.0) -> list:
    """View j of n: azimuth 2*pi*j/n in the x-z plane, fixed elevation, looking at the
    cube centre from dist_factor x the cube diagonal, up = +y."""
    nx, ny, nz = (float(d) for d in dims)
    c = (nx / 2, ny / 2, nz / 2)
    dist = dist_factor * math.sqrt(nx * nx + ny * ny + nz * nz)
    th = math.radians(elevation_deg)
    cams = []
    for j in range(n_views):
        ph = 2.0 * math.pi * j / n_views
        eye = (c[0] + dist * math.cos(th) * math.cos(ph), c[1] + dist * math.sin(th),
               c[2] + dist * math.cos(th) * math.sin(ph))
        cams.append(camera("persp", eye, c, (0.0, 1.0, 0.0), fovy_deg=fovy_deg))
    return cams


def random_cameras(dims, n: int, seed: int) -> list:
    """Random perspective viewpoints around the cube (serving requests)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = (float(d) for d in dims)
    c = (nx / 2, ny / 2, nz / 2)
    diag = math.sqrt(nx * nx + ny * ny + nz * nz)
    cams = []
    for _ in range(n):
        ph = rng.uniform(0, 2 * math.pi)
        th = rng.uniform(-0.6, 0.6)
        dist = rng.uniform(1.2, 2.0) * diag
        eye = (c[0] + dist * math.cos(th) * math.cos(ph), c[1] + dist * math.sin(th),
               c[2] + dist * math.cos(th) * math.sin(ph))
        cams.append(camera("persp", eye, c, (0.0, 1.0, 0.0), fovy_deg=float(rng.uniform(25, 40))))
    return cams


# --------------------------------------------------------------------------- transfer functions
def _ramp_rgb(u: np.ndarray) -> np.ndarray:
    return np.stack([u, 4.0 * u * (1.0 - u), 1.0 - u], axis=1)


def tf_sparse() -> np.ndarray:
    """256 RGBA (float32, colour not premultiplied): alpha 0 below u = 0.15, then a
    linear ramp to 0.8 at u = 1 -- noise is transparent, sources are opaque."""
    u = np.arange(256, dtype=np.float64) / 255.0
    a = np.where(u < 0.15, 0.0, 0.8 * (u - 0.15) / 0.85)
    return np.concatenate([_ramp_rgb(u), a[:, None]], axis=1).astype(np.float32)


def tf_dense() -> np.ndarray:
    """As tf_sparse with an alpha floor of 0.01 everywhere (early termination fires)."""
    t = tf_sparse().astype(np.float64)
    t[:, 3] = np.minimum(1.0, t[:, 3] + 0.01)
    return t.astype(np.float32)


def tf_constant(rgb, alpha: float) -> np.ndarray:
    t = np.empty((256, 4), dtype=np.float32)
    t[:, :3] = np.asarray(rgb, dtype=np.float32)
    t[:, 3] = np.float32(alpha)
    return t


def tf_random(seed: int) -> np.ndarray:
    """Seeded piecewise-linear transfer function (serving requests)."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(3, 8))
    xs = np.sort(np.concatenate([[0.0, 1.0], rng.uniform(0, 1, k)]))
    ys = rng.uniform(0, 1, (xs.size, 4))
    ys[:, 3] *= 0.6
    ys[0, 3] = 0.0
    u = np.arange(256) / 255.0
    t = np.stack([np.interp(u, xs, ys[:, c]) for c in range(4)], axis=1)
    return t.astype(np.float32)


# --------------------------------------------------------------------------- workloads
#: The five workloads, each with its seeded recipe.  Sizes follow the paper's
#: Table 1 range (4 GB .. 204 GB cubes); sources scale with volume.
WORKLOADS = {
    "small128": dict(dims=(128, 128, 128), n_sources=8, seed=1),
    "dvr1024": dict(dims=(1024, 1024, 1024), n_sources=2000, seed=2),
    "precision2048x2048x4096": dict(dims=(2048, 2048, 4096), n_sources=16000, seed=3),
    "ooc4096x4096x3072": dict(dims=(4096, 4096, 3072), n_sources=96000, seed=4),
}


def serving_stream(seed: int = 5, rate_hz: float = 200.0, duration_s: float = 60.0,
                   n_cubes: int = 64, sides=(256, 384, 512, 768, 1024)) -> dict:
    """Poisson request stream over a resident set of cubes (plain data only)."""
    rng = np.random.default_rng(seed)
    cubes = []
    for i in range(n_cubes):
        s = int(rng.choice(sides))
        cubes.append(dict(dims=(s, s, s), n_sources=max(1, int(8 * (s / 128) ** 3 // 8)),
                          seed=1000 + i, dtype=str(rng.choice(["f32", "bf16"]))))
    t = 0.0
    reqs = []
    sizes = [(512, 512), (1024, 1024), (1920, 1080)]
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        r = rng.uniform()
        kind = "dvr" if r < 0.5 else ("mip" if r < 0.8 else "stats")
        w, h = sizes[int(rng.integers(0, 3))]
        reqs.append(dict(t=t, kind=kind, cube=int(rng.integers(0, n_cubes)), width=w, height=h,
                         view_seed=int(rng.integers(0, 2**31)), tf_seed=int(rng.integers(0, 2**31))))
    return dict(cubes=cubes, requests=reqs)


class CgCube(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64), ("seed", ctypes.c_uint64),
                ("n_sources", ctypes.c_int32), ("B", ctypes.c_int32), ("calls", ctypes.c_int64)]


class BrickSource:
    """C brick provider of a generated cube for out-of-core uploads.

    ``fn`` is the address of ``cg_brick_source`` (int32 (*)(void *user, int64
    brick, int32 bx, int32 by, int32 bz, float *dst)), ``user`` the address of
    its cube record; the object must outlive every use of the pair.  ``calls``
    counts the bricks generated so far.  Generating through it needs no Python
    per brick.
    """

    def __init__(self, dims, n_sources: int, seed: int, brick: int):
        lib = _load()
        self.rec = CgCube(int(dims[0]), int(dims[1]), int(dims[2]), int(seed), int(n_sources), int(brick), 0)
        self.fn = ctypes.cast(lib.cg_brick_source, ctypes.c_void_p).value
        self.user = ctypes.addressof(self.rec)

    @property
    def calls(self) -> int:
        return int(self.rec.calls)

    def brick(self, b: int, nb) -> np.ndarray:
        """Brick b with halo as a (B+2)^3 float32 array (z, y, x)."""
        R = self.rec.B + 2
        out = np.empty((R, R, R), dtype=np.float32)
        bx, by, bz = b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])
        rc = _load().cg_brick_source(self.user, b, bx, by, bz, out.ctypes.data)
        if rc != 0:
            raise ValueError(f"cubegen: brick {b} failed")
        return out

