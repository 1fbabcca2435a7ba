"""The allocation-free statistics entry point (vrc_cube_stats_noalloc).

It exists for callers that must not allocate device memory when they ask for
statistics (latency-bound loops where cudaMalloc can stall the device, or
applications that keep all device memory in their own pool).  It must give the
same answer as vrc_cube_stats_async, call after call, while the library's
charged memory stays unchanged.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import cubegen

pytestmark = pytest.mark.gpu


def _read_stats(t):
    raw = t.cpu().numpy().tobytes()
    mn, mx, mean, std = np.frombuffer(raw[:32], dtype=np.float64)
    n, nnf = np.frombuffer(raw[32:48], dtype=np.uint64)
    return dict(min=mn, max=mx, mean=mean, std=std, n=int(n), n_nonfinite=int(nnf))


def test_noalloc_stats_match_async_on_two_calls():
    import paper_1111_6661_b300 as vrc
    lib = vrc.lib()
    ctx = vrc.Context(0)
    v = cubegen.generate((96, 80, 72), 6, 17)
    v[5, 6, 7] = np.nan                      # a non-finite voxel is skipped and counted
    cid = ctx.cube_upload(v, "f32", brick=32)
    nbins = 300
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    ref_out = torch.zeros(6, dtype=torch.float64, device="cuda")
    ref_hist = torch.zeros(nbins, dtype=torch.int64, device="cuda")
    ctx.cube_stats_async(cid, nbins, ref_out, ref_hist)
    torch.cuda.synchronize()
    ref = _read_stats(ref_out)
    used_before = ctx.memory()[0]

    for _ in range(2):
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        hist = torch.full((nbins,), 7, dtype=torch.int64, device="cuda")   # must be overwritten
        st = lib.vrc_cube_stats_noalloc(ctx.h, cid, nbins, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(hist.data_ptr()), stream)
        assert st == 0, lib.vrc_last_error(ctx.h)
        torch.cuda.synchronize()
        got = _read_stats(out)
        assert got["n"] == ref["n"] and got["n_nonfinite"] == ref["n_nonfinite"] == 1
        assert got["min"] == ref["min"] and got["max"] == ref["max"]
        assert abs(got["mean"] - ref["mean"]) <= 1e-9 * max(abs(ref["mean"]), ref["std"])
        assert abs(got["std"] - ref["std"]) <= 1e-9 * ref["std"]
        assert torch.equal(hist, ref_hist)
        assert ctx.memory()[0] == used_before          # nothing charged, nothing allocated

    # invalid arguments are refused before anything runs
    assert lib.vrc_cube_stats_noalloc(ctx.h, cid, -1, ctypes.c_void_p(out.data_ptr()), None, stream) == -1
    assert lib.vrc_cube_stats_noalloc(ctx.h, 999, 0, ctypes.c_void_p(out.data_ptr()), None, stream) == -5
    ctx.cube_free(cid)
    ctx.close()
