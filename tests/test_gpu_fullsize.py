"""Parity at full size, in the launch configuration the benchmark times.

The 1024^3 float32 cube of the DVR workload (N(0,1) noise + 2000 Gaussian
sources, seed 2, 256^3 bricks): the statistics pass with 4096 bins over all
2^30 voxels against the oracle in full (min/max and every histogram count
bit-exact, mean/std within 1e-9 relative), and the 32-view 1920x1080 DVR
orbit rendered in one persistent launch, checked on sampled pixels of every
view (a random set plus one full row) against the oracle pixel by pixel
(1e-4 absolute per RGBA channel; termination-fragile pixels inside the
oracle's bracket).  The empty-space-skipping variant and the slab march must
give the same image bit for bit on every pixel.
"""
import numpy as np
import pytest
import torch

import bench
import cubegen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

PIXELS_PER_VIEW = 512
# largest share of termination-fragile pixels allowed per view (see
# test_gpu_parity.FRAGILE_MAX); measured at most 3.21% over the 32 orbit views
FRAGILE_MAX = 0.035


@pytest.fixture(scope="module")
def full():
    import paper_1111_6661_b300 as vrc
    w = bench.workload("dvr1024")
    v, cams, tf = bench.make_inputs(w)
    ctx = vrc.Context(0)
    cid = ctx.cube_upload(v, w["storage"], brick=w["brick"])
    yield w, v, cams, tf, ctx, cid
    ctx.cube_free(cid)
    ctx.close()


def test_fullsize_stats(full):
    w, v, cams, tf, ctx, cid = full
    dstats = torch.empty(8, dtype=torch.float64, device="cuda")
    dhist = torch.empty(w["nbins"], dtype=torch.int64, device="cuda")
    ctx.cube_stats_async(cid, w["nbins"], dstats, dhist)
    torch.cuda.synchronize()
    s = dstats.cpu().numpy()
    n = dstats.cpu().view(torch.int64).numpy()[4:6]
    ref = oracle.stats(v)
    assert int(n[0]) == ref["n"] == v.size and int(n[1]) == 0
    assert s[0] == ref["min"] and s[1] == ref["max"]
    assert abs(s[2] - ref["mean"]) <= 1e-9 * max(abs(ref["mean"]), ref["std"]), (s[2], ref["mean"])
    assert abs(s[3] - ref["std"]) <= 1e-9 * ref["std"], (s[3], ref["std"])
    h = oracle.histogram(v, ref["min"], ref["max"], w["nbins"])
    assert np.array_equal(dhist.cpu().numpy().astype(np.uint64), h)
    assert int(h.sum()) == v.size


def test_fullsize_median(full):
    w, v, cams, tf, ctx, cid = full
    m = ctx.cube_median(cid)
    k = (v.size - 1) // 2
    assert m == float(np.partition(v.reshape(-1), k)[k])


def test_fullsize_dvr_orbit(full):
    import paper_1111_6661_b300 as vrc
    w, v, cams, tf, ctx, cid = full
    info = ctx.cube_info(cid)
    W, H = w["W"], w["H"]
    rc = vrc.raycfg(W, H, w["step"], "trilinear")
    out = torch.empty((len(cams), H, W, 4), dtype=torch.float32, device="cuda")
    ctx.render_dvr(cid, cams, rc, tf, w["term"], out=out)
    torch.cuda.synchronize()
    assert ctx.last_render_samples() > 0
    rng = np.random.default_rng(12)
    img = out.cpu().numpy().reshape(len(cams), -1, 4).astype(np.float64)
    nonzero = 0
    for i, cam in enumerate(cams):
        row = int(rng.integers(0, H))
        pix = np.unique(np.concatenate([rng.choice(W * H, size=PIXELS_PER_VIEW, replace=False),
                                        row * W + np.arange(W)]))
        r = oracle.render(v, cam, W, H, w["step"], "trilinear", "dvr", tf=tf, vmin=info["vmin"],
                          vmax=info["vmax"], term=w["term"], pixels=pix)
        got = img[i, pix]
        d = np.abs(got - r["out"]).max(axis=1)
        ok = d <= 1e-4
        inside = np.all((got >= r["lo"] - 1e-4) & (got <= r["hi"] + 1e-4), axis=1)
        ok |= r["fragile"] & inside
        frac = float(r["fragile"].mean())
        print(f"view {i}: fragile fraction {frac:.4f} ({int(r['fragile'].sum())} of {r['fragile'].size})")
        assert ok.all(), (i, int((~ok).sum()), float(d.max()), f"fragile fraction {frac:.4f}")
        assert frac <= FRAGILE_MAX, (i, f"fragile fraction {frac:.4f}")
        nonzero += int((r["out"][:, 3] > 0).sum())
    assert nonzero > 0   # the sampled pixels see sources, not only background

    # empty-space skipping and the slab march: the same image, bit for bit, on
    # every pixel of every view
    n_fused = ctx.last_render_samples()
    for rc2 in (vrc.raycfg(W, H, w["step"], "trilinear", skip_empty=True),
                vrc.raycfg(W, H, w["step"], "trilinear", path="slab")):
        out2 = torch.empty_like(out)
        ctx.render_dvr(cid, cams, rc2, tf, w["term"], out=out2)
        torch.cuda.synchronize()
        assert torch.equal(out, out2)
        assert ctx.last_render_samples() == n_fused


def test_fullsize_native_nearest_mip(full):
    """Orthographic nearest MIP along z at native resolution (1024x1024,
    step 1): every pixel equals its column maximum, bit for bit, and every
    voxel is sampled once."""
    import paper_1111_6661_b300 as vrc
    w, v, cams, tf, ctx, cid = full
    NX, NY, NZ = w["dims"]
    img = ctx.render_mip(cid, [cubegen.ortho_z_camera(w["dims"])], vrc.raycfg(NX, NY, 1.0, "nearest"))
    torch.cuda.synchronize()
    assert ctx.last_render_samples() == v.size
    assert np.array_equal(img[0].cpu().numpy(), v.max(axis=0))


def test_fullsize_trilinear_mip(full):
    import paper_1111_6661_b300 as vrc
    w, v, cams, tf, ctx, cid = full
    W, H = w["W"], w["H"]
    views = [cams[0], cams[11]]
    img = ctx.render_mip(cid, views, vrc.raycfg(W, H, w["step"], "trilinear"))
    torch.cuda.synchronize()
    got = img.cpu().numpy().reshape(len(views), -1).astype(np.float64)
    rng = np.random.default_rng(13)
    for i, cam in enumerate(views):
        pix = rng.choice(W * H, size=PIXELS_PER_VIEW, replace=False)
        r = oracle.render(v, cam, W, H, w["step"], "trilinear", "mip", pixels=pix)
        err = np.abs(got[i, pix] - r["out"]) / np.maximum(np.abs(r["out"]), 1.0)
        assert err.max() <= 1e-5, (i, err.max())


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_fullsize_precision_storage(full, dtype):
    """The bench cube stored as bf16 / fp8 e4m3 (per-brick scale) in 256^3
    bricks: statistics over all 2^30 stored values against the oracle on the
    dequantised cube (min/max, histogram and median exact, mean/std 1e-9), the
    native-resolution nearest MIP equal to the stored column maxima, sampled
    pixels of DVR and trilinear MIP renders at the fp32 tolerances."""
    import paper_1111_6661_b300 as vrc
    w, v, cams, tf, ctx, _ = full
    B = w["brick"]
    cid = ctx.cube_upload(v, dtype, brick=B)
    try:
        dq = oracle.dequantize(v, dtype, B)
        s, h = ctx.cube_stats(cid, 1024)
        ref = oracle.stats(dq)
        assert s["min"] == ref["min"] and s["max"] == ref["max"] and s["n"] == ref["n"]
        assert abs(s["mean"] - ref["mean"]) <= 1e-9 * max(abs(ref["mean"]), ref["std"])
        assert abs(s["std"] - ref["std"]) <= 1e-9 * ref["std"]
        assert np.array_equal(h, oracle.histogram(dq, ref["min"], ref["max"], 1024))
        k = (dq.size - 1) // 2
        assert ctx.cube_median(cid) == float(np.partition(dq.reshape(-1), k)[k])
        # native-resolution orthographic nearest MIP (row-group kernel): the stored column maxima
        NX, NY, NZ = w["dims"]
        nat = ctx.render_mip(cid, [cubegen.ortho_z_camera(w["dims"])], vrc.raycfg(NX, NY, 1.0, "nearest"))
        torch.cuda.synchronize()
        assert ctx.last_render_path() == "rows" and ctx.last_render_samples() == v.size
        assert np.array_equal(nat[0].cpu().numpy(), dq.max(axis=0))
        del dq, nat
        info = ctx.cube_info(cid)
        W, H = w["W"], w["H"]
        views = [cams[3], cams[20]]
        rc = vrc.raycfg(W, H, w["step"], "trilinear")
        dvr = ctx.render_dvr(cid, views, rc, tf, w["term"])
        mip = ctx.render_mip(cid, views, rc)
        torch.cuda.synchronize()
        dvr = dvr.cpu().numpy().reshape(len(views), -1, 4).astype(np.float64)
        mip = mip.cpu().numpy().reshape(len(views), -1).astype(np.float64)
        rng = np.random.default_rng(21)
        for i, cam in enumerate(views):
            pix = rng.choice(W * H, size=PIXELS_PER_VIEW, replace=False)
            kw = dict(pixels=pix, dtype=dtype, brick=B)
            r = oracle.render(v, cam, W, H, w["step"], "trilinear", "dvr", tf=tf, vmin=info["vmin"],
                              vmax=info["vmax"], term=w["term"], **kw)
            got = dvr[i, pix]
            d = np.abs(got - r["out"]).max(axis=1)
            inside = np.all((got >= r["lo"] - 1e-4) & (got <= r["hi"] + 1e-4), axis=1)
            assert ((d <= 1e-4) | (r["fragile"] & inside)).all(), (i, float(d.max()))
            r = oracle.render(v, cam, W, H, w["step"], "trilinear", "mip", **kw)
            err = np.abs(mip[i, pix] - r["out"]) / np.maximum(np.abs(r["out"]), 1.0)
            assert err.max() <= 1e-5, (i, err.max())
    finally:
        ctx.cube_free(cid)
