"""Python binding of the B300 cube ray-casting / statistics library (include/vrc.h).

Argument marshalling only: every step of the path runs in the CUDA kernels of
libvrc.so.  PyTorch provides device memory and streams.  There is no CPU
fallback; if libvrc.so is missing the import of the binding fails loudly.

Names follow the C ABI: ``Context.cube_upload`` calls ``vrc_cube_upload`` and
so on.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _vrc
from ._vrc import COPY, DTYPES, INJECT, PATH_NAMES, PATHS, SAMPLING

__all__ = ["VrcError", "Context", "raycfg", "camera_struct", "lib"]


class VrcError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{_vrc.STATUS.get(status, status)}: {msg}")


def lib():
    return _vrc.load()


def camera_struct(cam: dict) -> _vrc.vrc_camera:
    c = _vrc.vrc_camera()
    c.kind = int(cam["kind"])
    for a in range(3):
        c.eye[a] = cam["eye"][a]
        c.center[a] = cam["center"][a]
        c.up[a] = cam["up"][a]
    c.fovy_deg = cam.get("fovy_deg", 30.0)
    c.ortho_height = cam.get("ortho_height", 1.0)
    return c


def raycfg(width: int, height: int, step: float, sampling: str = "trilinear", opacity_correction: bool = False,
           path: str = "fused", tile=(0, 0), skip_empty: bool = False) -> _vrc.vrc_raycfg:
    return _vrc.vrc_raycfg(int(width), int(height), float(step), SAMPLING[sampling], int(opacity_correction),
                           PATHS[path], int(tile[0]), int(tile[1]), int(skip_empty), 0)


def _stream_ptr(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _cams(cams):
    if isinstance(cams, dict):
        cams = [cams]
    arr = (_vrc.vrc_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_struct(c)
    return arr, len(cams)


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, n_streams: int = 0, max_inflight: int = 0):
        self._lib = lib()
        cfg = _vrc.vrc_config(device, n_streams, max_inflight, 0, hbm_budget_bytes)
        h = ctypes.c_void_p()
        self._check(self._lib.vrc_create(ctypes.byref(h), ctypes.byref(cfg)), ctx=False)
        self.h = h
        self.device = device

    # ------------------------------------------------------------ plumbing
    def _check(self, st: int, ctx: bool = True, ok=(0,)):
        if st not in ok:
            msg = self._lib.vrc_last_error(self.h).decode() if ctx else ""
            raise VrcError(st, msg)
        return st

    def close(self):
        if getattr(self, "h", None):
            self._check(self._lib.vrc_destroy(self.h), ctx=False)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def memory(self):
        u, b = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.vrc_memory(self.h, ctypes.byref(u), ctypes.byref(b)))
        return u.value, b.value

    def launch_count(self) -> int:
        return int(self._lib.vrc_launch_count(self.h))

    def debug_inject(self, what: str, nth: int = 1):
        self._check(self._lib.vrc_debug_inject(self.h, INJECT[what], nth))

    # ------------------------------------------------------------ cubes
    def cube_upload(self, src, storage: str = "f32", brick: int = 0, stream=None, render_copy: str = "auto") -> int:
        """src: float32 array (sz, sy, sx) -- numpy (host) or torch tensor (host or cuda).
        render_copy: "auto" (made when it fits), "required" (VRC_E_NOMEM when it
        does not fit) or "none"."""
        import torch
        if isinstance(src, np.ndarray):
            assert src.dtype == np.float32 and src.flags.c_contiguous and src.ndim == 3
            ptr, on_dev, shape = src.ctypes.data, 0, src.shape
        else:
            assert src.dtype == torch.float32 and src.is_contiguous() and src.dim() == 3
            ptr, on_dev, shape = src.data_ptr(), int(src.is_cuda), tuple(src.shape)
        cid = ctypes.c_int64()
        self._check(self._lib.vrc_cube_upload(self.h, ctypes.c_void_p(ptr), on_dev, shape[2], shape[1], shape[0],
                                              DTYPES[storage] | COPY[render_copy], brick, _stream_ptr(stream),
                                              ctypes.byref(cid)))
        return cid.value

    def cube_register(self, src: np.ndarray, storage: str = "f32", brick: int = 0, render_copy: str = "auto") -> int:
        """Register a host cube (float32 numpy array (sz, sy, sx)) that the
        library makes resident only while it is needed; the array is kept
        referenced until cube_free.  bf16 / fp8 cubes are packed once here and
        load from their packed host copy afterwards."""
        assert isinstance(src, np.ndarray) and src.dtype == np.float32 and src.flags.c_contiguous and src.ndim == 3
        cid = ctypes.c_int64()
        self._check(self._lib.vrc_cube_register(self.h, ctypes.c_void_p(src.ctypes.data), src.shape[2], src.shape[1],
                                                src.shape[0], DTYPES[storage] | COPY[render_copy], brick,
                                                ctypes.byref(cid)))
        if not hasattr(self, "_sources"):
            self._sources = {}
        self._sources[cid.value] = src
        return cid.value

    def residency(self) -> dict:
        """Registered cubes resident now, uploads and evictions so far."""
        r, l, e = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self._lib.vrc_residency(self.h, ctypes.byref(r), ctypes.byref(l), ctypes.byref(e)))
        return dict(resident=r.value, loads=l.value, evictions=e.value)

    def cube_create_streamed(self, dims, brick: int, n_host_bricks: int, ring_bricks: int = 0) -> int:
        cid = ctypes.c_int64()
        self._check(self._lib.vrc_cube_create_streamed(self.h, dims[0], dims[1], dims[2], brick, n_host_bricks,
                                                       ring_bricks, ctypes.byref(cid)))
        self._out_of_core = getattr(self, "_out_of_core", set()) | {cid.value}
        return cid.value

    def cube_upload_streamed(self, dims, brick: int, source, n_host_bricks: int, ring_bricks: int = 0,
                             storage: str = "f32") -> int:
        """Out-of-core cube whose bricks come from `source`: either a pair
        (C function address, user address) of a vrc_brick_source_fn, or a
        Python callable (brick, bx, by, bz) -> float32 array of (B+2)^3 values
        (z, y, x) holding the brick and its clamp-to-edge halo.  storage: the
        type the host cache and the device ring keep the bricks in."""
        if callable(source):
            R = int(brick) + 2

            def _cb(user, b, bx, by, bz, dst, _f=source):
                try:
                    a = np.ctypeslib.as_array(dst, shape=(R * R * R,))
                    a[:] = np.asarray(_f(int(b), int(bx), int(by), int(bz)), dtype=np.float32).reshape(-1)
                    return 0
                except Exception:   # reported to the library as a provider failure
                    return 1
            fn = _vrc.BRICK_SOURCE_FN(_cb)
            fn_ptr, user = ctypes.cast(fn, ctypes.c_void_p), None
        else:
            fn, (fn_ptr, user) = source, source
        cid = ctypes.c_int64()
        self._check(self._lib.vrc_cube_upload_streamed(self.h, ctypes.c_void_p(fn_ptr.value if hasattr(fn_ptr, "value")
                                                                               else fn_ptr),
                                                       ctypes.c_void_p(user), dims[0], dims[1], dims[2],
                                                       DTYPES[storage], brick, n_host_bricks, ring_bricks,
                                                       ctypes.byref(cid)))
        # the provider (and its closure) must outlive the cube
        if not hasattr(self, "_sources"):
            self._sources = {}
        self._sources[cid.value] = fn
        self._out_of_core = getattr(self, "_out_of_core", set()) | {cid.value}
        return cid.value

    def cube_put_brick(self, cube_id: int, slot: int, brick_with_halo: np.ndarray):
        b = np.ascontiguousarray(brick_with_halo, dtype=np.float32)
        self._check(self._lib.vrc_cube_put_brick(self.h, cube_id, slot, b.ctypes.data))

    def cube_free(self, cube_id: int):
        self._check(self._lib.vrc_cube_free(self.h, cube_id))
        getattr(self, "_sources", {}).pop(cube_id, None)

    def cube_free_async(self, cube_id: int, stream=None):
        """Release once the work issued on `stream` so far has completed."""
        self._check(self._lib.vrc_cube_free_async(self.h, cube_id, _stream_ptr(stream)))

    def cube_info(self, cube_id: int) -> dict:
        dims = (ctypes.c_int64 * 3)()
        B, st, nb, by = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        mn, mx, tb = ctypes.c_float(), ctypes.c_float(), ctypes.c_int64()
        self._check(self._lib.vrc_cube_info(self.h, cube_id, dims, ctypes.byref(B), ctypes.byref(st),
                                            ctypes.byref(nb), ctypes.byref(by), ctypes.byref(mn), ctypes.byref(mx),
                                            ctypes.byref(tb)))
        return dict(dims=tuple(dims), brick=B.value, storage={v: k for k, v in DTYPES.items()}[st.value],
                    n_bricks=nb.value, bytes=by.value, vmin=mn.value, vmax=mx.value, render_copy_bytes=tb.value)

    def cube_read_brick(self, cube_id: int, brick: int) -> np.ndarray:
        """Stored form of one brick: array (R, R, P) of float32 / uint16 (bf16
        bits) / uint8 (e4m3 codes), R = B + 2 planes and rows (local -1..B),
        local x at element O + x of a row (O = 32 / element size; out-of-core
        cubes 16 / element size)."""
        info = self.cube_info(cube_id)
        B = info["brick"]
        dt = {"f32": np.float32, "bf16": np.uint16, "fp8": np.uint8}[info["storage"]]
        es = np.dtype(dt).itemsize
        align = 16 if cube_id in getattr(self, "_out_of_core", ()) else 32
        R, P = B + 2, B + 2 * (align // es)
        out = np.empty((R, R, P), dtype=dt)
        self._check(self._lib.vrc_cube_read_brick(self.h, cube_id, brick, ctypes.c_void_p(out.ctypes.data),
                                                  out.nbytes))
        return out

    # ------------------------------------------------------------ statistics
    def cube_stats(self, cube_id: int, nbins: int = 0, stream=None):
        out = _vrc.vrc_stats()
        hist = np.zeros(max(nbins, 1), dtype=np.uint64)
        self._check(self._lib.vrc_cube_stats(self.h, cube_id, nbins, ctypes.byref(out),
                                             ctypes.c_void_p(hist.ctypes.data), _stream_ptr(stream)))
        s = dict(min=out.min, max=out.max, mean=out.mean, std=out.std, n=out.n, n_nonfinite=out.n_nonfinite)
        return s, hist[:nbins]

    def cube_stats_async(self, cube_id: int, nbins: int, dev_out, dev_hist, stream=None):
        """dev_out: cuda tensor of >= 48 bytes; dev_hist: cuda int64 tensor [nbins] or None."""
        self._check(self._lib.vrc_cube_stats_async(self.h, cube_id, nbins, ctypes.c_void_p(dev_out.data_ptr()),
                                                   ctypes.c_void_p(dev_hist.data_ptr() if dev_hist is not None else 0),
                                                   _stream_ptr(stream)))

    def cube_median(self, cube_id: int, stream=None) -> float:
        out = ctypes.c_double()
        self._check(self._lib.vrc_cube_median(self.h, cube_id, ctypes.byref(out), _stream_ptr(stream)))
        return out.value

    # ------------------------------------------------------------ rendering
    def render_mip(self, cube_id: int, cams, rc: _vrc.vrc_raycfg, out=None, stream=None):
        import torch
        arr, n = _cams(cams)
        if out is None:
            out = torch.empty((n, rc.height, rc.width), dtype=torch.float32, device=f"cuda:{self.device}")
        assert out.is_cuda and out.dtype == torch.float32 and out.numel() >= n * rc.height * rc.width
        self._check(self._lib.vrc_render_mip(self.h, cube_id, arr, n, ctypes.byref(rc),
                                             ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def render_dvr(self, cube_id: int, cams, rc: _vrc.vrc_raycfg, tf: np.ndarray, term_alpha: float = 0.99,
                   out=None, stream=None):
        import torch
        arr, n = _cams(cams)
        tfa = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1)
        assert tfa.size == 1024
        if out is None:
            out = torch.empty((n, rc.height, rc.width, 4), dtype=torch.float32, device=f"cuda:{self.device}")
        assert out.is_cuda and out.dtype == torch.float32 and out.numel() >= n * rc.height * rc.width * 4
        self._check(self._lib.vrc_render_dvr(self.h, cube_id, arr, n, ctypes.byref(rc),
                                             ctypes.c_void_p(tfa.ctypes.data), term_alpha,
                                             ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def last_render_samples(self, evaluated: bool = False):
        """Lattice samples of the last render (and, with evaluated=True, the
        samples actually fetched as a second value)."""
        n, e = ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self._lib.vrc_last_render_samples(self.h, ctypes.byref(n), ctypes.byref(e)))
        return (n.value, e.value) if evaluated else n.value

    def last_render_path(self) -> str:
        """Path the last render took: fused (texture gathers), fused_ldg (global
        loads), sortlast, streamed, zerocopy or slab."""
        p = ctypes.c_int32()
        self._check(self._lib.vrc_last_render_path(self.h, ctypes.byref(p)))
        return PATH_NAMES[p.value]

    def last_render_bricks(self):
        """(traversed, culled) distinct bricks of the last sort-last render."""
        t, c = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.vrc_last_render_bricks(self.h, ctypes.byref(t), ctypes.byref(c)))
        return t.value, c.value

    def composite(self, front, back, mode: str = "dvr", out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(front)
        n = front.numel() // (4 if mode == "dvr" else 1)
        self._check(self._lib.vrc_composite(self.h, ctypes.c_void_p(front.data_ptr()),
                                            ctypes.c_void_p(back.data_ptr()), ctypes.c_void_p(out.data_ptr()), n,
                                            0 if mode == "mip" else 1, _stream_ptr(stream)))
        return out

    # ------------------------------------------------------------ batching
    def graph_create(self, cube_id: int, cams, rc, out, tf=None, term_alpha: float = 0.99):
        arr, n = _cams(cams)
        g = ctypes.c_void_p()
        tfp = None
        if tf is not None:
            self._graph_tf = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1)
            tfp = ctypes.c_void_p(self._graph_tf.ctypes.data)
        self._check(self._lib.vrc_graph_create(self.h, cube_id, arr, n, ctypes.byref(rc), tfp, term_alpha,
                                               ctypes.c_void_p(out.data_ptr()), ctypes.byref(g)))
        return g

    def graph_launch(self, g, stream=None):
        self._check(self._lib.vrc_graph_launch(g, _stream_ptr(stream)))

    def graph_destroy(self, g):
        self._check(self._lib.vrc_graph_destroy(g))

    def autotune(self, cube_id: int, cams, rc, out, tf=None, term_alpha: float = 0.99, stream=None,
                 brick_search: bool = False, step_tolerance: float = 0.0) -> dict:
        """Ray tile and grid search (vrc_autotune); with brick_search or a step
        tolerance, vrc_autotune_cube (brick edges {64, 128, 256}, faster steps
        within the tolerance)."""
        arr, n = _cams(cams)
        res = _vrc.vrc_tuning()
        tfp = None
        if tf is not None:
            tfa = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1)
            tfp = ctypes.c_void_p(tfa.ctypes.data)
        if brick_search or step_tolerance > 0:
            self._check(self._lib.vrc_autotune_cube(self.h, cube_id, arr, n, ctypes.byref(rc), tfp, term_alpha,
                                                    ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream),
                                                    1 if brick_search else 0, step_tolerance, ctypes.byref(res)))
        else:
            self._check(self._lib.vrc_autotune(self.h, cube_id, arr, n, ctypes.byref(rc), tfp, term_alpha,
                                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream), ctypes.byref(res)))
        return dict(tile=(res.tile_w, res.tile_h), ctas_per_sm=res.ctas_per_sm, brick=res.brick, step=res.step,
                    best_ms=res.best_ms, default_ms=res.default_ms, step_max_abs_diff=res.step_max_abs_diff)

    # ------------------------------------------------------------ serving
    def submit(self, kind: str, cube_id: int, cam=None, rc=None, tf=None, term_alpha: float = 0.99, nbins: int = 0,
               out=None) -> int:
        req = _vrc.vrc_request()
        req.kind = {"mip": 0, "dvr": 1, "stats": 2}[kind]
        req.nbins = nbins
        req.cube_id = cube_id
        if cam is not None:
            req.cam = camera_struct(cam)
        if rc is not None:
            req.rc = rc
        if tf is not None:
            tfa = np.ascontiguousarray(tf, dtype=np.float32).reshape(-1)
            ctypes.memmove(req.tf_rgba, tfa.ctypes.data, 4096)
        req.term_alpha = term_alpha
        req.out = ctypes.c_void_p(out.data_ptr() if out is not None else 0)
        t = ctypes.c_uint64()
        self._check(self._lib.vrc_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """Returns a result dict, or None while pending (timeout_ms == 0)."""
        res = _vrc.vrc_result()
        st = self._lib.vrc_poll(self.h, ticket, ctypes.byref(res), timeout_ms)
        if st == _vrc.VRC_PENDING:
            return None
        self._check(st)
        s = res.stats
        return dict(status=res.status, queue_ms=res.queue_ms, latency_ms=res.latency_ms, samples=res.samples,
                    path=PATH_NAMES.get(res.path, res.path), memory_wait_ms=res.memory_wait_ms,
                    cube_loaded=bool(res.cube_loaded),
                    stats=dict(min=s.min, max=s.max, mean=s.mean, std=s.std, n=s.n, n_nonfinite=s.n_nonfinite))
