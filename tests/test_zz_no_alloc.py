"""The allocation-free statistics entry point (vrc_cube_stats_noalloc).

It exists for callers that must not allocate device memory when they ask for
statistics (latency-bound loops where cudaMalloc can stall the device, or
applications that keep all device memory in their own pool).  Called first on
a fresh context, it must charge and allocate nothing, and give the same answer
as vrc_cube_stats_async, call after call, for every storage type and every
histogram path (none, shared-memory counters, global counters).  This file is
collected last on purpose.
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


@pytest.mark.parametrize("nbins", [0, 300, 20000])
@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_noalloc_stats_match_async_on_two_calls(dtype, nbins):
    import paper_1111_6661_b300 as vrc
    lib = vrc.lib()
    ctx = vrc.Context(0)
    v = cubegen.generate((96, 80, 72), 6, 17)
    v[5, 6, 7] = np.nan                      # a non-finite voxel is skipped and counted
    cid = ctx.cube_upload(v, dtype, brick=32)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    used_before = ctx.memory()[0]

    # the allocation-free call comes first on this context, so the context's
    # own scratch buffer does not exist yet: any allocation would show up
    got = []
    for _ in range(2):
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        hist = torch.full((max(nbins, 1),), 7, dtype=torch.int64, device="cuda")   # must be overwritten
        st = lib.vrc_cube_stats_noalloc(ctx.h, cid, nbins, ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(hist.data_ptr() if nbins else 0), stream)
        assert st == 0, lib.vrc_last_error(ctx.h)
        torch.cuda.synchronize()
        assert ctx.memory()[0] == used_before          # nothing charged, nothing allocated
        got.append((_read_stats(out), hist[:nbins].clone()))

    ref_out = torch.zeros(6, dtype=torch.float64, device="cuda")
    ref_hist = torch.zeros(max(nbins, 1), dtype=torch.int64, device="cuda")
    ctx.cube_stats_async(cid, nbins, ref_out, ref_hist if nbins else None)
    torch.cuda.synchronize()
    ref = _read_stats(ref_out)
    for g, h in got:
        assert g["n"] == ref["n"] and g["n_nonfinite"] == ref["n_nonfinite"] == 1
        assert g["min"] == ref["min"] and g["max"] == ref["max"]
        assert abs(g["mean"] - ref["mean"]) <= 1e-9 * max(abs(ref["mean"]), ref["std"])
        assert abs(g["std"] - ref["std"]) <= 1e-9 * ref["std"]
        assert torch.equal(h, ref_hist[:nbins])
        if nbins:
            assert int(h.sum()) == ref["n"]

    # invalid arguments are refused before anything runs
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    assert lib.vrc_cube_stats_noalloc(ctx.h, cid, -1, ctypes.c_void_p(out.data_ptr()), None, stream) == -1
    assert lib.vrc_cube_stats_noalloc(ctx.h, 999, 0, ctypes.c_void_p(out.data_ptr()), None, stream) == -5
    ctx.cube_free(cid)
    ctx.close()
