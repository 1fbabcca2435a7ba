"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances: min/max, histogram counts, nearest-sample MIP and the median are
bit-exact; mean/std within 1e-9 relative; trilinear MIP within 1e-5 relative
(floor 1 on the magnitude); DVR within 1e-4 absolute per premultiplied RGBA
channel (pixels whose accumulated alpha crosses the termination threshold
within binary32 rounding may stop one sample earlier or later, and must then
lie inside the oracle's bracket of admissible results).
"""
import numpy as np
import pytest
import torch

import cubegen
import oracle

pytestmark = pytest.mark.gpu

F32MAX = float(np.finfo(np.float32).max)


@pytest.fixture(scope="module")
def ctx():
    import paper_1111_6661_b300 as vrc
    c = vrc.Context(0)
    yield c
    c.close()


def vrcmod():
    import paper_1111_6661_b300 as vrc
    return vrc


def ragged_cube():
    return cubegen.generate((37, 29, 23), 4, 21)


def stored(v, dtype, B):
    return v if dtype == "f32" else oracle.dequantize(v, dtype, B)


def check_stats(s, h, ref_v, nbins):
    ref = oracle.stats(ref_v)
    assert s["n"] == ref["n"] and s["n_nonfinite"] == ref["n_nonfinite"]
    assert s["min"] == ref["min"] and s["max"] == ref["max"]
    scale = max(abs(ref["mean"]), ref["std"], 1e-30)
    assert abs(s["mean"] - ref["mean"]) <= 1e-9 * scale, (s["mean"], ref["mean"])
    assert abs(s["std"] - ref["std"]) <= 1e-9 * max(ref["std"], 1e-300) or ref["std"] == s["std"]
    if nbins:
        assert np.array_equal(h, oracle.histogram(ref_v, ref["min"], ref["max"], nbins))


# ------------------------------------------------------------------ statistics
@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("case", ["cfg128", "ragged"])
def test_stats_parity(ctx, dtype, case, cube128):
    v, B, nbins = (cube128, 128, 256) if case == "cfg128" else (ragged_cube(), 16, 100)
    cid = ctx.cube_upload(v, dtype, brick=B)
    s, h = ctx.cube_stats(cid, nbins)
    check_stats(s, h, stored(v, dtype, B), nbins)
    ctx.cube_free(cid)


@pytest.mark.parametrize("nbins", [1, 4096, 20000])
def test_stats_bins_and_device_source(ctx, nbins, cube128):
    t = torch.from_numpy(cube128).cuda()
    cid = ctx.cube_upload(t, "f32", brick=32)
    s, h = ctx.cube_stats(cid, nbins)
    check_stats(s, h, cube128, nbins)
    ctx.cube_free(cid)


def test_stats_closed_forms(ctx):
    c = np.full((20, 18, 17), 2.5, np.float32)
    cid = ctx.cube_upload(c, "f32", brick=16)
    s, h = ctx.cube_stats(cid, 8)
    assert s["mean"] == 2.5 and s["std"] == 0 and h[0] == c.size
    ctx.cube_free(cid)
    r = np.arange(64 * 32 * 16, dtype=np.float32).reshape(16, 32, 64)
    cid = ctx.cube_upload(r, "f32", brick=16)
    s, h = ctx.cube_stats(cid, 256)
    n = r.size
    assert abs(s["mean"] - (n - 1) / 2) <= 1e-12 * n
    assert abs(s["std"] ** 2 - (n * n - 1) / 12) <= 1e-9 * (n * n / 12)
    check_stats(s, h, r, 256)
    ctx.cube_free(cid)


def test_stats_nonfinite(ctx):
    v = ragged_cube().copy()
    v[3, 4, 5] = np.nan
    v[7, 1, 0] = np.inf
    v[0, 0, 36] = -np.inf
    cid = ctx.cube_upload(v, "f32", brick=16)
    s, h = ctx.cube_stats(cid, 32)
    assert s["n_nonfinite"] == 3
    check_stats(s, h, v, 32)
    ctx.cube_free(cid)
    vrc = vrcmod()
    allnan = np.full((16, 16, 16), np.nan, np.float32)
    cid = ctx.cube_upload(allnan, "f32", brick=16)
    with pytest.raises(vrc.VrcError, match="NONFINITE"):
        ctx.cube_stats(cid, 4)
    ctx.cube_free(cid)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_median_exact(ctx, dtype, cube128):
    for v, B in [(cube128, 64), (ragged_cube(), 16), (np.arange(1000, dtype=np.float32).reshape(10, 10, 10) - 500, 16)]:
        cid = ctx.cube_upload(v, dtype, brick=B)
        assert ctx.cube_median(cid) == oracle.median(stored(v, dtype, B))
        ctx.cube_free(cid)


def test_median_special_values(ctx):
    """Non-finite voxels are skipped, -0 and +0 are one value, ties and an
    even count take the lower median, every digit of the key is exercised."""
    rng = np.random.default_rng(4)
    v = rng.standard_normal((33, 31, 29)).astype(np.float32)
    flat = v.reshape(-1)
    flat[::97] = np.nan
    flat[5::211] = np.inf
    flat[7::313] = -np.inf
    flat[11::17] = -0.0
    flat[13::19] = 0.0
    flat[20:40] = flat[41]                       # ties across the median region
    for B in (16, 32):
        cid = ctx.cube_upload(v, "f32", brick=B)
        assert ctx.cube_median(cid) == oracle.median(v)
        ctx.cube_free(cid)
    w = np.array([3.0, -1.0, 2.0, 7.0], np.float32).reshape(1, 2, 2)   # even count: lower median 2.0
    cid = ctx.cube_upload(w, "f32", brick=16)
    assert ctx.cube_median(cid) == 2.0
    ctx.cube_free(cid)


def test_median_candidates_kept_or_not(ctx):
    """Float32 medians keep the keys that share the median's leading 12-bit
    digit for their last pass; more than 2^26 such keys (here 84 M voxels in
    [1, 1.125), one digit) make the last pass read the cube again.  Both give
    the oracle's lower median."""
    rng = np.random.default_rng(9)
    v = (1.0 + 0.124 * rng.random((320, 512, 512))).astype(np.float32)
    cid = ctx.cube_upload(v, "f32", brick=256)
    assert ctx.cube_median(cid) == oracle.median(v)
    ctx.cube_free(cid)
    w = v[:64, :256, :256].copy()             # 4 M candidates: kept
    cid = ctx.cube_upload(w, "f32", brick=64)
    assert ctx.cube_median(cid) == oracle.median(w)
    ctx.cube_free(cid)


def sampled_rows_mask(shape, B, esize, stride=61):
    """Voxels of a cube (dims multiples of B, esize bytes per stored value)
    that the median's sample reads: chunks of 256 16-byte vectors, i.e.
    4096 / (esize B) consecutive rows (z_local, y_local) of one brick, every
    stride-th chunk in brick order."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    b = ((z // B) * (ny // B) + y // B) * (nx // B) + x // B
    rows_per_chunk = 4096 // (esize * B)
    chunk = b * (B * B // rows_per_chunk) + ((z % B) * B + y % B) // rows_per_chunk
    return chunk % stride == 0


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_median_bracket(ctx, dtype):
    """Cubes of at least 2^22 voxels: a sample of the rows bounds the median's
    leading digit, and one pass over the cube keeps the keys of the bounded
    bins.  A generated cube (the bracket holds the median), a cube with many
    ties, and a cube whose sampled rows hold values far above the rest (the
    bracket misses; the passes read the cube) give the oracle's lower median."""
    v = cubegen.generate((256, 256, 128), 40, 7)
    rng = np.random.default_rng(12)
    ties = np.round(rng.standard_normal((128, 256, 256)) * 4).astype(np.float32)
    skew = rng.standard_normal((128, 256, 256)).astype(np.float32)
    m = sampled_rows_mask(skew.shape, 64, 4 if dtype == "f32" else 2)
    assert 0.01 < m.mean() < 0.02
    skew[m] = 1000.0 + rng.random(int(m.sum())).astype(np.float32)
    for w in (v, ties, skew):
        cid = ctx.cube_upload(w, dtype, brick=64)
        assert ctx.cube_median(cid) == oracle.median(stored(w, dtype, 64))
        assert ctx.cube_median(cid) == oracle.median(stored(w, dtype, 64))   # the call again
        ctx.cube_free(cid)


# ------------------------------------------------------------------ rendering
def render_check_mip(ctx, v, cid, cams, W, H, step, sampling, dtype="f32", B=0, path="fused"):
    vrc = vrcmod()
    rc = vrc.raycfg(W, H, step, sampling, path=path)
    img = ctx.render_mip(cid, cams, rc)
    torch.cuda.synchronize()
    got = img.cpu().numpy().reshape(len(cams), -1).astype(np.float64)
    for i, cam in enumerate(cams):
        r = oracle.render(v, cam, W, H, step, sampling, "mip", dtype=dtype, brick=B if dtype != "f32" else 0)
        if sampling == "nearest":
            assert np.array_equal(got[i], r["out"]), (i, np.abs(got[i] - r["out"]).max())
        else:
            err = np.abs(got[i] - r["out"]) / np.maximum(np.abs(r["out"]), 1.0)
            assert err.max() <= 1e-5, (i, err.max())
    return got


# Largest share of termination-fragile pixels allowed in one image: pixels
# whose stopping sample a binary32 evaluation could move (the oracle's alpha
# window, see oracle.render); they are checked against the oracle's bracket
# instead of its exact-index result.  Measured at most 1.87% in these tests.
FRAGILE_MAX = 0.02


def check_dvr(got, r, tol=1e-4):
    d = np.abs(got - r["out"]).max(axis=1)
    ok = d <= tol
    inside = np.all((got >= r["lo"] - tol) & (got <= r["hi"] + tol), axis=1)
    ok |= r["fragile"] & inside
    frac = float(r["fragile"].mean())
    print(f"fragile fraction {frac:.4f} ({int(r['fragile'].sum())} of {r['fragile'].size})")
    assert ok.all(), (int((~ok).sum()), float(d.max()), f"fragile fraction {frac:.4f}")
    assert frac <= FRAGILE_MAX, f"fragile fraction {frac:.4f}"


def render_check_dvr(ctx, v, cid, cams, W, H, step, tf, term=0.99, dtype="f32", B=0, path="fused", opc=False,
                     sampling="trilinear"):
    vrc = vrcmod()
    rc = vrc.raycfg(W, H, step, sampling, opacity_correction=opc, path=path)
    img = ctx.render_dvr(cid, cams, rc, tf, term)
    torch.cuda.synchronize()
    info = ctx.cube_info(cid)
    got = img.cpu().numpy().reshape(len(cams), -1, 4).astype(np.float64)
    for i, cam in enumerate(cams):
        r = oracle.render(v, cam, W, H, step, sampling, "dvr", tf=tf, vmin=info["vmin"], vmax=info["vmax"], term=term,
                          opacity_correction=opc, dtype=dtype, brick=B if dtype != "f32" else 0)
        check_dvr(got[i], r)
    return got


def test_axis_aligned_mip_cfg128(ctx, cube128):
    """128^3 cube, orthographic along z, 256x256, step 1: nearest is bit-exact
    and equals the column maximum; trilinear within 1e-5."""
    cid = ctx.cube_upload(cube128, "f32", brick=128)
    cam = cubegen.ortho_z_camera((128, 128, 128))
    got = render_check_mip(ctx, cube128, cid, [cam], 256, 256, 1.0, "nearest")
    col = cube128.max(axis=0).astype(np.float64)
    assert np.array_equal(got[0].reshape(256, 256), np.repeat(np.repeat(col, 2, 0), 2, 1))
    render_check_mip(ctx, cube128, cid, [cam], 256, 256, 1.0, "trilinear")
    ctx.cube_free(cid)


@pytest.mark.parametrize("B", [16, 32, 64])
@pytest.mark.parametrize("sampling", ["nearest", "trilinear"])
def test_perspective_mip(ctx, B, sampling, cube128):
    v = cube128[:70, :50, :90].copy()   # ragged against every brick size
    dims = (90, 50, 70)
    cid = ctx.cube_upload(v, "f32", brick=B)
    cams = cubegen.orbit_cameras(dims, 3) + cubegen.random_cameras(dims, 2, B)
    render_check_mip(ctx, v, cid, cams, 61, 47, 0.5, sampling)
    ctx.cube_free(cid)


@pytest.mark.parametrize("tfname", ["sparse", "dense"])
def test_perspective_dvr(ctx, tfname, cube128):
    v = cube128[:70, :50, :90].copy()
    dims = (90, 50, 70)
    cid = ctx.cube_upload(v, "f32", brick=32)
    tf = cubegen.tf_sparse() if tfname == "sparse" else cubegen.tf_dense()
    cams = cubegen.orbit_cameras(dims, 2) + cubegen.random_cameras(dims, 2, 4)
    render_check_dvr(ctx, v, cid, cams, 64, 48, 0.5, tf)
    ctx.cube_free(cid)


def test_dvr_variants(ctx, cube128):
    v = cube128[:40, :40, :40].copy()
    cid = ctx.cube_upload(v, "f32", brick=16)
    cams = cubegen.orbit_cameras((40, 40, 40), 2)
    render_check_dvr(ctx, v, cid, cams, 32, 32, 0.5, cubegen.tf_dense(), term=2.0)        # no termination
    render_check_dvr(ctx, v, cid, cams, 32, 32, 0.7, cubegen.tf_random(3), opc=True)      # opacity correction
    render_check_dvr(ctx, v, cid, cams, 32, 32, 1.0, cubegen.tf_dense(), sampling="nearest")
    ctx.cube_free(cid)


def test_uniform_alpha_closed_form_gpu(ctx):
    v = np.ones((40, 8, 8), np.float32)
    cid = ctx.cube_upload(v, "f32", brick=16)
    vrc = vrcmod()
    for a in (0.05, 0.3):
        tf = cubegen.tf_constant((0.2, 0.5, 1.0), a)
        cam = cubegen.ortho_z_camera((8, 8, 40))
        img = ctx.render_dvr(cid, [cam], vrc.raycfg(8, 8, 1.0), tf, 2.0).cpu().numpy().reshape(-1, 4)
        A = 1 - (1 - np.float64(np.float32(a))) ** 40
        assert np.allclose(img[:, 3], A, atol=1e-5)
        assert np.allclose(img[:, :3], np.array([0.2, 0.5, 1.0]) * A, atol=1e-5)
    ctx.cube_free(cid)


@pytest.mark.parametrize("mode", ["mip", "dvr"])
def test_sortlast_matches_oracle_and_fused(ctx, mode, cube128):
    v = cube128[:70, :50, :90].copy()
    dims = (90, 50, 70)
    cid = ctx.cube_upload(v, "f32", brick=16)
    cams = cubegen.orbit_cameras(dims, 2) + cubegen.random_cameras(dims, 1, 7)
    cams.append(cubegen.camera("persp", (40.3, 22.1, 31.7), (0, 0, 0), (0, 1, 0), fovy_deg=70))  # eye inside
    if mode == "mip":
        a = render_check_mip(ctx, v, cid, cams, 48, 40, 0.5, "trilinear", path="sortlast")
        b = render_check_mip(ctx, v, cid, cams, 48, 40, 0.5, "trilinear", path="fused")
        assert np.array_equal(a, b)
    else:
        tf = cubegen.tf_dense()
        a = render_check_dvr(ctx, v, cid, cams, 48, 40, 0.5, tf, path="sortlast")
        b = render_check_dvr(ctx, v, cid, cams, 48, 40, 0.5, tf, path="fused")
        assert np.abs(a - b).max() <= 1e-4
    ctx.cube_free(cid)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_precision_storage(ctx, dtype, cube128):
    """BF16 / FP8 bricks against the oracle on the same stored (dequantised)
    bricks at the fp32 tolerances; the error against the original fp32 cube is
    reported by the benchmark."""
    v = cube128[:64, :64, :64].copy()
    B = 32
    cid = ctx.cube_upload(v, dtype, brick=B)
    cams = cubegen.orbit_cameras((64, 64, 64), 2)
    render_check_mip(ctx, v, cid, cams, 40, 40, 0.5, "nearest", dtype=dtype, B=B)
    render_check_mip(ctx, v, cid, cams, 40, 40, 0.5, "trilinear", dtype=dtype, B=B)
    render_check_dvr(ctx, v, cid, cams, 40, 40, 0.5, cubegen.tf_dense(), dtype=dtype, B=B)
    ctx.cube_free(cid)


def test_multiview_batch_equals_single(ctx, cube128):
    vrc = vrcmod()
    cid = ctx.cube_upload(cube128, "f32", brick=64)
    cams = cubegen.orbit_cameras((128, 128, 128), 4)
    rc = vrc.raycfg(50, 30, 0.5)
    tf = cubegen.tf_sparse()
    batch = ctx.render_dvr(cid, cams, rc, tf).cpu()
    for i, c in enumerate(cams):
        one = ctx.render_dvr(cid, [c], rc, tf).cpu()
        assert torch.equal(one[0], batch[i])
    # tile shapes do not change any pixel
    for tile in [(8, 32), (32, 8)]:
        t = ctx.render_dvr(cid, cams, vrc.raycfg(50, 30, 0.5, tile=tile), tf).cpu()
        assert torch.equal(t, batch)
    ctx.cube_free(cid)


def test_graph_and_autotune(ctx, cube128):
    vrc = vrcmod()
    cid = ctx.cube_upload(cube128, "f32", brick=64)
    cams = cubegen.orbit_cameras((128, 128, 128), 3)
    rc = vrc.raycfg(64, 48, 0.5)
    tf = cubegen.tf_dense()
    ref = ctx.render_dvr(cid, cams, rc, tf).clone()
    out = torch.zeros_like(ref)
    g = ctx.graph_create(cid, cams, rc, out, tf=tf)
    for _ in range(2):
        out.zero_()
        ctx.graph_launch(g)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    ctx.graph_destroy(g)
    res = ctx.autotune(cid, cams, rc, out, tf=tf)
    assert res["tile"] in [(8, 32), (16, 16), (32, 8)] and res["ctas_per_sm"] >= 1
    assert res["best_ms"] <= res["default_ms"] + 1e-9
    again = ctx.render_dvr(cid, cams, rc, tf)
    assert torch.equal(again, ref)
    ctx.cube_free(cid)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_autotune_brick_edge_and_step(ctx, cube128, dtype):
    """The batching form's autotuner: the cube re-packed on the device at brick
    edges 64 and 128 (the stored values are kept exactly), the fastest edge
    replacing its storage under the same id; images and statistics are the
    same at every edge, and they still match the oracle.  A faster step is
    taken only within the caller's image tolerance."""
    vrc = vrcmod()
    v = cube128[:, :, :120].copy()          # 120 x 128 x 128: ragged along x at edge 64 and 128
    cid = ctx.cube_upload(v, dtype, brick=32)
    cams = cubegen.orbit_cameras((120, 128, 128), 2)
    rc = vrc.raycfg(64, 48, 0.5)
    tf = cubegen.tf_dense()
    ref = ctx.render_dvr(cid, cams, rc, tf).clone()
    s0, h0 = ctx.cube_stats(cid, 100)
    out = torch.zeros_like(ref)
    res = ctx.autotune(cid, cams, rc, out, tf=tf, brick_search=True)
    assert res["brick"] in (32, 64, 128) and ctx.cube_info(cid)["brick"] == res["brick"]
    assert res["step"] == rc.step and res["step_max_abs_diff"] == 0.0
    assert res["best_ms"] <= res["default_ms"] + 1e-9
    assert torch.equal(ctx.render_dvr(cid, cams, rc, tf), ref)
    s1, h1 = ctx.cube_stats(cid, 100)
    assert s1["min"] == s0["min"] and s1["max"] == s0["max"] and np.array_equal(h0, h1)
    assert abs(s1["mean"] - s0["mean"]) <= 1e-12 * s0["std"] and abs(s1["std"] - s0["std"]) <= 1e-12 * s0["std"]
    vv = v if dtype == "f32" else oracle.dequantize(v, dtype)
    render_check_dvr(ctx, vv, cid, cams[:1], 64, 48, 0.5, tf)
    # every edge gives the same image: re-pack at each one through the tuner's trial path
    for B in (64, 128):
        other = ctx.cube_upload(v, dtype, brick=B)
        assert torch.equal(ctx.render_dvr(other, cams, rc, tf), ref)
        ctx.cube_free(other)
    # step: a tolerance of 0 never changes it; a loose one may take a faster step within it
    res = ctx.autotune(cid, cams, rc, out, tf=tf, step_tolerance=1.0)
    assert res["step"] >= rc.step and res["step_max_abs_diff"] <= 1.0
    res2 = ctx.autotune(cid, cams, rc, out, tf=tf, step_tolerance=1e-9)
    assert res2["step"] == rc.step or res2["step_max_abs_diff"] <= 1e-9
    ctx.cube_free(cid)


def test_composite_api(ctx):
    rng = np.random.default_rng(1)
    a = rng.uniform(0, 1, (300, 1))
    f = np.concatenate([rng.uniform(0, 1, (300, 3)) * a, a], 1)
    a = rng.uniform(0, 1, (300, 1))
    b = np.concatenate([rng.uniform(0, 1, (300, 3)) * a, a], 1)
    ft, bt = torch.tensor(f, dtype=torch.float32).cuda(), torch.tensor(b, dtype=torch.float32).cuda()
    out = ctx.composite(ft, bt, "dvr").cpu().numpy()
    ref = oracle.composite(ft.cpu().numpy(), bt.cpu().numpy(), "dvr")
    assert np.abs(out - ref).max() <= 1e-6
    x, y = torch.randn(77).cuda(), torch.randn(77).cuda()
    assert torch.equal(ctx.composite(x, y, "mip"), torch.maximum(x, y))


# ------------------------------------------------------------------ errors
def test_error_codes(ctx, cube128):
    vrc = vrcmod()
    with pytest.raises(vrc.VrcError, match="BADID"):
        ctx.cube_stats(12345, 4)
    with pytest.raises(vrc.VrcError, match="INVAL"):
        ctx.cube_upload(cube128, "f32", brick=24)
    cid = ctx.cube_upload(cube128, "f32", brick=64)
    with pytest.raises(vrc.VrcError, match="INVAL"):
        ctx.render_mip(cid, [cubegen.ortho_z_camera((128, 128, 128))], vrc.raycfg(0, 10, 1.0))
    bad = dict(cubegen.ortho_z_camera((128, 128, 128)))
    bad["up"] = [0.0, 0.0, 1.0]   # parallel to the view direction
    with pytest.raises(vrc.VrcError, match="INVAL"):
        ctx.render_mip(cid, [bad], vrc.raycfg(8, 8, 1.0))
    with pytest.raises(vrc.VrcError, match="INVAL"):
        ctx.cube_stats(cid, 70000)
    ctx.cube_free(cid)
    # more than 2^22 samples per ray: diagonal 5793 voxels at step 1e-3 (checked
    # before anything is read, so the streamed cube needs no bricks)
    big = (4096, 4096, 64)
    sid = ctx.cube_create_streamed(big, 256, 1, 2)
    with pytest.raises(vrc.VrcError, match=r"2\^22"):
        ctx.render_mip(sid, [cubegen.ortho_z_camera(big)], vrc.raycfg(8, 8, 1e-3))
    ctx.cube_free(sid)


def test_budget_and_injected_allocation_failure():
    vrc = vrcmod()
    small = vrc.Context(0, hbm_budget_bytes=4 << 20)
    v = np.zeros((128, 128, 128), np.float32)
    with pytest.raises(vrc.VrcError, match="NOMEM"):
        small.cube_upload(v, "f32", brick=64)   # 8.6 MB of bricks > 4 MiB
    assert small.memory()[0] == 0               # nothing leaked on the failure path
    small.close()
    c = vrc.Context(0)
    c.debug_inject("alloc", 2)
    with pytest.raises(vrc.VrcError, match="NOMEM"):
        c.cube_upload(v[:32, :32, :32].copy(), "f32", brick=16)
    cid = c.cube_upload(v[:32, :32, :32].copy(), "f32", brick=16)   # next call succeeds
    c.cube_free(cid)
    assert c.memory()[0] == 0 or c.memory()[0] > 0  # scratch may stay allocated
    c.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_texture_gather_equals_global_loads(ctx, dtype, cube128):
    """The fused renderer reads trilinear footprints with 2x2 texture gathers
    from per-brick layered arrays; the same lerps on the same stored values
    must reproduce the 8-global-load variant bit for bit."""
    vrc = vrcmod()
    v = cube128[:70, :50, :90].copy()
    dims = (90, 50, 70)
    cid = ctx.cube_upload(v, dtype, brick=32)
    assert ctx.cube_info(cid)["render_copy_bytes"] > 0     # the gather path is really taken
    c = (45.0, 25.0, 35.0)
    axis_views = [cubegen.camera("persp", (c[0], c[1], -200), c, (0, 1, 0)),     # rays along z
                  cubegen.camera("persp", (-250, c[1], c[2]), c, (0, 1, 0)),     # rays along x
                  cubegen.camera("persp", (c[0], 300, c[2]), c, (0, 0, 1))]      # rays along y
    cams = cubegen.orbit_cameras(dims, 3) + axis_views + [
        cubegen.camera("persp", (40.3, 22.1, 31.7), (0, 0, 0), (0, 1, 0), fovy_deg=70)]
    tf = cubegen.tf_dense()
    a = ctx.render_dvr(cid, cams, vrc.raycfg(64, 48, 0.5, path="fused"), tf).cpu()
    b = ctx.render_dvr(cid, cams, vrc.raycfg(64, 48, 0.5, path="fused_ldg"), tf).cpu()
    assert torch.equal(a, b)
    a = ctx.render_mip(cid, cams, vrc.raycfg(64, 48, 0.5, path="fused")).cpu()
    b = ctx.render_mip(cid, cams, vrc.raycfg(64, 48, 0.5, path="fused_ldg")).cpu()
    assert torch.equal(a, b)
    ctx.cube_free(cid)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_empty_space_skipping_is_exact(ctx, dtype, cube128):
    """skip_empty skips samples whose 8^3 macro-cell cannot change the result
    (transparent under the TF for DVR, below the ray's running max for MIP);
    the image must be bit-identical and fewer samples fetched."""
    vrc = vrcmod()
    v = cube128[:96, :80, :112].copy()
    dims = (112, 80, 96)
    cid = ctx.cube_upload(v, dtype, brick=32)
    cams = cubegen.orbit_cameras(dims, 3) + cubegen.random_cameras(dims, 2, 11)
    for tf in (cubegen.tf_sparse(), cubegen.tf_random(4)):
        a = ctx.render_dvr(cid, cams, vrc.raycfg(72, 56, 0.5), tf).cpu()
        n0, e0 = ctx.last_render_samples(evaluated=True)
        b = ctx.render_dvr(cid, cams, vrc.raycfg(72, 56, 0.5, skip_empty=True), tf).cpu()
        n1, e1 = ctx.last_render_samples(evaluated=True)
        assert torch.equal(a, b)
        assert n0 == n1 == e0 and e1 <= e0
    tf = cubegen.tf_sparse()
    _, e1 = ctx.render_dvr(cid, cams, vrc.raycfg(72, 56, 0.5, skip_empty=True), tf), None
    n1, e1 = ctx.last_render_samples(evaluated=True)
    assert e1 < 0.5 * n1          # the sparse TF leaves most of the noise transparent
    a = ctx.render_mip(cid, cams, vrc.raycfg(72, 56, 0.5)).cpu()
    b = ctx.render_mip(cid, cams, vrc.raycfg(72, 56, 0.5, skip_empty=True)).cpu()
    assert torch.equal(a, b)
    ctx.cube_free(cid)


def test_cached_allocations_reused_and_trimmed(cube128):
    """Freed cubes return their device blocks and render-copy arrays to the
    context's cache; a cube of the same shape reuses them and renders the same
    image, and a small budget still admits a differently shaped cube (the
    cache gives way)."""
    vrc = vrcmod()
    c = vrc.Context(0)
    cams = cubegen.orbit_cameras((128, 128, 128), 2)
    rc = vrc.raycfg(48, 40, 0.5)
    cid = c.cube_upload(cube128, "f32", brick=64)
    assert c.cube_info(cid)["render_copy_bytes"] > 0
    a = c.render_mip(cid, cams, rc).cpu()
    d = c.render_dvr(cid, cams, rc, cubegen.tf_dense()).cpu()
    used = c.memory()[0]
    c.cube_free(cid)
    cid = c.cube_upload(cube128, "f32", brick=64)
    assert torch.equal(a, c.render_mip(cid, cams, rc).cpu())
    assert torch.equal(d, c.render_dvr(cid, cams, rc, cubegen.tf_dense()).cpu())
    assert c.memory()[0] == used
    c.cube_free(cid)
    c.close()
    small = vrc.Context(0, hbm_budget_bytes=32 << 20)
    for brick in (64, 32, 64, 32):
        sid = small.cube_upload(cube128, "f32", brick=brick)
        st, _ = small.cube_stats(sid, 16)
        assert st["n"] == 128 ** 3
        small.cube_free(sid)
        assert small.memory()[0] <= 32 << 20
    small.close()


def test_free_async_is_stream_ordered(cube128):
    """vrc_cube_free_async: the id is gone at once, the render already issued
    on the stream still reads the cube, and its memory is reused by the next
    upload of the same shape; under a budget that holds one cube, the next
    upload waits for the released one instead of failing."""
    vrc = vrcmod()
    c = vrc.Context(0)
    cams = cubegen.orbit_cameras((128, 128, 128), 3)
    rc = vrc.raycfg(64, 48, 0.5)
    tf = cubegen.tf_dense()
    cid = c.cube_upload(cube128, "f32", brick=64)
    ref = c.render_dvr(cid, cams, rc, tf).cpu()
    used_one = c.memory()[0]
    s = torch.cuda.Stream()
    for _ in range(3):
        out = torch.empty((len(cams), 48, 64, 4), dtype=torch.float32, device="cuda")
        c.render_dvr(cid, cams, rc, tf, out=out, stream=s)
        c.cube_free_async(cid, stream=s)
        with pytest.raises(vrc.VrcError):
            c.cube_info(cid)
        cid = c.cube_upload(cube128, "f32", brick=64)   # may reuse the released blocks
        s.synchronize()
        assert torch.equal(out.cpu(), ref)
    torch.cuda.synchronize()
    other = c.cube_upload(cube128[:64].copy(), "f32", brick=64)   # any allocation reaps completed releases
    assert c.memory()[0] < 2 * used_one
    c.cube_free(other)
    # a budget that holds one cube and the next one's pool but not its staging
    # copy: the second upload waits for the stream-ordered release (no render
    # copies fit this budget; those renders read the bricks, same image)
    pool = c.cube_info(cid)["bytes"]
    c.cube_free(cid)
    c.close()
    small = vrc.Context(0, hbm_budget_bytes=int(2.2 * pool))
    a = small.cube_upload(cube128, "f32", brick=64)
    out = torch.empty((len(cams), 48, 64, 4), dtype=torch.float32, device="cuda")
    small.render_dvr(a, cams, rc, tf, out=out, stream=s)
    small.cube_free_async(a, stream=s)
    b = small.cube_upload(cube128, "f32", brick=64)
    assert torch.equal(small.render_dvr(b, cams, rc, tf).cpu(), ref)
    s.synchronize()
    assert torch.equal(out.cpu(), ref)
    small.cube_free(b)
    small.close()


# ------------------------------------------------------------------ slab path
def axis_cameras(dims):
    """Views whose rays run mainly along +-x, +-y and +-z (every principal
    axis and direction of the slab march), perspective and orthographic, and
    one with the eye inside the cube."""
    nx, ny, nz = dims
    c = (nx / 2, ny / 2, nz / 2)
    d = 2.5 * max(dims)
    cams = []
    for a in range(3):
        for sgn in (1, -1):
            eye = list(c)
            eye[a] += sgn * d
            eye[(a + 1) % 3] += 0.21 * d   # a little off-axis
            up = (0.0, 0.0, 1.0) if a == 1 else (0.0, 1.0, 0.0)
            cams.append(cubegen.camera("persp", eye, c, up, fovy_deg=30))
    cams.append(cubegen.camera("ortho", (c[0] + 0.3, c[1] - 0.2, -d), c, (0, 1, 0), ortho_height=1.3 * ny))
    cams.append(cubegen.camera("persp", (0.6 * nx, 0.45 * ny, 0.5 * nz), (0, 0, 0), (0, 1, 0), fovy_deg=80))
    return cams


@pytest.mark.parametrize("mode", ["mip", "dvr"])
def test_slab_path_matches_oracle_and_fused(ctx, mode, cube128):
    """The slab march (tiles staged in shared memory by TMA) against the
    oracle at the stated tolerances, and bit-identical to the fused texture
    renderer, on a ragged cube, for every principal axis and direction."""
    v = cube128[:70, :50, :90].copy()
    dims = (90, 50, 70)
    cid = ctx.cube_upload(v, "f32", brick=32)
    cams = axis_cameras(dims) + cubegen.orbit_cameras(dims, 3) + cubegen.random_cameras(dims, 3, 17)
    W, H = 75, 53   # ragged against the 16x16 tiles
    if mode == "mip":
        a = render_check_mip(ctx, v, cid, cams, W, H, 0.5, "trilinear", path="slab")
        n_slab = ctx.last_render_samples()
        b = render_check_mip(ctx, v, cid, cams, W, H, 0.5, "trilinear", path="fused")
        assert np.array_equal(a, b)
    else:
        tf = cubegen.tf_dense()
        a = render_check_dvr(ctx, v, cid, cams, W, H, 0.5, tf, path="slab")
        n_slab = ctx.last_render_samples()
        b = render_check_dvr(ctx, v, cid, cams, W, H, 0.5, tf, path="fused")
        assert np.array_equal(a, b)
    assert n_slab == ctx.last_render_samples()
    ctx.cube_free(cid)


def test_slab_path_large_tiles_and_steps(ctx, cube128):
    """Bigger cube than one staged box in every direction, coarse and fine
    steps, sparse TF with early termination off and on."""
    vrc = vrcmod()
    cid = ctx.cube_upload(cube128, "f32", brick=64)
    dims = (128, 128, 128)
    cams = axis_cameras(dims)[:4] + cubegen.orbit_cameras(dims, 2)
    for step, tf, term in [(0.37, cubegen.tf_sparse(), 0.99), (1.0, cubegen.tf_dense(), 2.0),
                           (0.5, cubegen.tf_random(5), 0.99)]:
        rc_s = vrc.raycfg(96, 80, step, "trilinear", path="slab")
        rc_f = vrc.raycfg(96, 80, step, "trilinear", path="fused")
        a = ctx.render_dvr(cid, cams, rc_s, tf, term)
        b = ctx.render_dvr(cid, cams, rc_f, tf, term)
        torch.cuda.synchronize()
        assert torch.equal(a, b), step
    got = a.cpu().numpy().reshape(len(cams), -1, 4).astype(np.float64)
    info = ctx.cube_info(cid)
    rng = np.random.default_rng(3)
    for i in (0, 5):
        pix = rng.choice(96 * 80, size=600, replace=False)
        r = oracle.render(cube128, cams[i], 96, 80, 0.5, "trilinear", "dvr", tf=cubegen.tf_random(5),
                          vmin=info["vmin"], vmax=info["vmax"], term=0.99, pixels=pix)
        check_dvr(got[i, pix], r)
    ctx.cube_free(cid)


def test_slab_wait_runs_out_and_context_survives(ctx, cube128):
    """The slab renderer's wait for its staging copy is bounded: with the
    copies withheld (host-side injection; nothing faults) the render reports
    VRC_E_TIMEOUT within seconds, and the context renders correctly after."""
    import time
    vrc = vrcmod()
    v = cube128[:64, :64, :64].copy()
    cid = ctx.cube_upload(v, "f32", brick=32)
    cams = cubegen.orbit_cameras((64, 64, 64), 2)
    rc = vrc.raycfg(48, 40, 0.5, "trilinear", path="slab")
    ref = ctx.render_mip(cid, cams, rc).cpu()
    ctx.debug_inject("slab_wait", 1)
    t0 = time.time()
    ctx.render_mip(cid, cams, rc)
    with pytest.raises(vrc.VrcError) as err:
        ctx.last_render_samples()
    assert err.value.status == -4   # VRC_E_TIMEOUT
    assert time.time() - t0 < 30
    assert torch.equal(ctx.render_mip(cid, cams, rc).cpu(), ref)
    ctx.last_render_samples()
    ctx.cube_free(cid)


def test_slab_path_rejects_what_it_does_not_cover(ctx, cube128):
    vrc = vrcmod()
    v = cube128[:32, :32, :32].copy()
    cam = cubegen.orbit_cameras((32, 32, 32), 1)
    cid = ctx.cube_upload(v, "bf16", brick=16)
    with pytest.raises(vrc.VrcError):
        ctx.render_mip(cid, cam, vrc.raycfg(16, 16, 0.5, "trilinear", path="slab"))
    ctx.cube_free(cid)
    cid = ctx.cube_upload(v, "f32", brick=16)
    for rc in (vrc.raycfg(16, 16, 0.5, "nearest", path="slab"),
               vrc.raycfg(16, 16, 0.5, "trilinear", path="slab", skip_empty=True)):
        with pytest.raises(vrc.VrcError):
            ctx.render_mip(cid, cam, rc)
    ctx.cube_free(cid)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_axis_aligned_nearest_mip_every_direction(ctx, dtype):
    """Orthographic nearest MIP along +-x, +-y and +-z (rays with two zero
    direction components take the fixed-index loop), ragged cube and bricks,
    step 1 and 0.7: every pixel equals the oracle's bit for bit."""
    v = cubegen.generate((48, 40, 36), 5, 61)
    dims = (48, 40, 36)
    B = 16
    cid = ctx.cube_upload(v, dtype, brick=B)
    c = [d / 2 for d in dims]
    cams = []
    for axis in range(3):
        for sign in (1.0, -1.0):
            eye = list(c)
            eye[axis] = c[axis] - sign * 2 * dims[axis]
            up = [0.0, 1.0, 0.0] if axis != 1 else [0.0, 0.0, 1.0]
            cams.append(cubegen.camera("ortho", eye, c, up, ortho_height=float(max(dims))))
    for step in (1.0, 0.7):
        render_check_mip(ctx, v, cid, cams, 44, 44, step, "nearest", dtype=dtype, B=B)
    ctx.cube_free(cid)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_row_group_nearest_mip(ctx, dtype):
    """Orthographic nearest MIP along +-z and +-y at native resolution takes the
    row-group kernel (8 rays of an image row per thread, one vector load per
    sample): image x along +x and along -x, a view shifted by 3 voxels
    (no group aligned: every group takes the per-ray loop), a width that
    leaves a ragged last group, fp8 scales changing along the ray.  Every pixel
    equals the oracle's bit for bit, and a view that does not qualify
    (perspective) in the same call keeps the per-ray kernel."""
    vrc = vrcmod()
    dims = (60, 48, 40)
    B = 16
    v = cubegen.generate(dims, 6, 67)
    # special columns: all values <= 0 with -0 and +0 (a zero maximum: the
    # per-ray loop decides), a NaN, an infinity (fp8 stores it as NaN)
    v[:, 5, 7] = -np.abs(v[:, 5, 7]) - 1.0
    v[3, 5, 7], v[9, 5, 7] = 0.0, -0.0
    v[:, 6, 9] = -np.abs(v[:, 6, 9]) - 1.0
    v[4, 6, 9] = -0.0
    v[10, 6, 8] = np.nan
    v[11, 7, 9] = np.inf
    cid = ctx.cube_upload(v, dtype, brick=B)
    nx, ny, nz = dims
    c = (nx / 2, ny / 2, nz / 2)
    zview = [cubegen.ortho_z_camera(dims),
             cubegen.camera("ortho", (c[0], c[1], nz + 5.0), c, (0, -1, 0), ortho_height=float(ny)),   # x reversed
             cubegen.camera("ortho", (c[0] + 3.0, c[1], -5.0), (c[0] + 3.0, c[1], 0.0), (0, -1, 0),
                            ortho_height=float(ny))]                                                  # shifted
    yview = [cubegen.camera("ortho", (c[0], -5.0, c[2]), c, (0, 0, 1), ortho_height=float(nz)),
             cubegen.camera("ortho", (c[0], ny + 5.0, c[2]), c, (0, 0, 1), ortho_height=float(nz))]
    for cams, W, H in ((zview, nx, ny), (yview, nx, nz)):
        for step in (1.0, 0.7):
            render_check_mip(ctx, v, cid, cams, W, H, step, "nearest", dtype=dtype, B=B)
            assert ctx.last_render_path() == "rows"
            assert ctx.last_render_samples() > 0
    # 48-pixel-wide z views over x = 0 .. 47 (every group full and aligned), image x along +x and -x
    cam48 = [cubegen.camera("ortho", (24.0, c[1], -5.0), (24.0, c[1], 0.0), (0, -1, 0), ortho_height=float(ny)),
             cubegen.camera("ortho", (24.0, c[1], nz + 5.0), (24.0, c[1], 0.0), (0, -1, 0), ortho_height=float(ny))]
    got = render_check_mip(ctx, v, cid, cam48, 48, ny, 1.0, "nearest", dtype=dtype, B=B)
    assert ctx.last_render_path() == "rows"
    assert np.array_equal(got[0].reshape(ny, 48), got[1].reshape(ny, 48)[:, ::-1])
    mixed = [zview[0], cubegen.orbit_cameras(dims, 4)[1]]
    render_check_mip(ctx, v, cid, mixed, nx, ny, 1.0, "nearest", dtype=dtype, B=B)
    assert ctx.last_render_path() == "fused_ldg"
    ctx.cube_free(cid)
