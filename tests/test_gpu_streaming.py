"""Out-of-core rendering: bricks (plus halo) in pinned host memory streamed to a
device ring on a side stream, per-wavefront partial images composited in
visibility order.  Checked against the resident renders and the oracle."""
import numpy as np
import pytest
import torch

import cubegen
import oracle

pytestmark = pytest.mark.gpu


def brick_with_halo(v, B, b, nb):
    bx, by, bz = b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])
    idx = [np.clip(np.arange(o * B - 1, o * B + B + 1), 0, n - 1) for o, n in zip((bz, by, bx), v.shape)]
    return np.ascontiguousarray(v[np.ix_(*idx)])


def make_streamed(ctx, v, B, n_host=None, ring=8, source=None):
    dims = (v.shape[2], v.shape[1], v.shape[0])
    nb = [(d + B - 1) // B for d in dims]
    total = nb[0] * nb[1] * nb[2]
    n_host = n_host or total
    cid = ctx.cube_create_streamed(dims, B, n_host, ring)
    for slot in range(n_host):
        b = slot if source is None else source(slot)
        ctx.cube_put_brick(cid, slot, brick_with_halo(v, B, b, nb))
    return cid, total


@pytest.fixture(scope="module")
def ctx():
    import paper_1111_6661_b300 as vrc
    c = vrc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("ring", [2, 8])
def test_streamed_matches_resident_and_oracle(ctx, cube128, ring):
    import paper_1111_6661_b300 as vrc
    v = cube128[:64, :48, :80].copy()
    dims = (80, 48, 64)
    sid, _ = make_streamed(ctx, v, 16, ring=ring)
    rid = ctx.cube_upload(v, "f32", brick=16)
    cams = cubegen.orbit_cameras(dims, 2) + [cubegen.camera("persp", (30.2, 20.5, 31.7), (0, 0, 0), (0, 1, 0),
                                                            fovy_deg=70)]
    rc = vrc.raycfg(40, 32, 0.5)
    a = ctx.render_mip(sid, cams, rc).cpu()
    b = ctx.render_mip(rid, cams, rc).cpu()
    assert torch.equal(a, b)
    tf = cubegen.tf_dense()
    a = ctx.render_dvr(sid, cams, rc, tf).cpu().numpy().reshape(len(cams), -1, 4).astype(np.float64)
    b = ctx.render_dvr(rid, cams, rc, tf).cpu().numpy().reshape(len(cams), -1, 4)
    assert np.abs(a - b).max() <= 1e-4
    info = ctx.cube_info(sid)
    assert info["vmin"] == float(v.min()) and info["vmax"] == float(v.max())
    for i, cam in enumerate(cams):
        r = oracle.render(v, cam, 40, 32, 0.5, "trilinear", "dvr", tf=tf, vmin=info["vmin"], vmax=info["vmax"])
        d = np.abs(a[i] - r["out"]).max(axis=1)
        ok = (d <= 1e-4) | (r["fragile"] & np.all((a[i] >= r["lo"] - 1e-4) & (a[i] <= r["hi"] + 1e-4), axis=1))
        assert ok.all()
    ctx.cube_free(sid)
    ctx.cube_free(rid)


def test_aliased_host_slots(ctx, cube128):
    """n_host_bricks < bricks: logical brick b reads host slot b % n.  The render
    must equal that of a cube whose every brick b holds slot (b % n)'s data."""
    import paper_1111_6661_b300 as vrc
    v = cube128[:48, :48, :48].copy()
    dims = (48, 48, 48)
    K = 5
    aid, total = make_streamed(ctx, v, 16, n_host=K)
    fid, _ = make_streamed(ctx, v, 16, n_host=None, source=lambda b: b % K)
    cams = cubegen.orbit_cameras(dims, 2)
    rc = vrc.raycfg(32, 32, 0.5)
    tf = cubegen.tf_sparse()
    assert torch.equal(ctx.render_dvr(aid, cams, rc, tf).cpu(), ctx.render_dvr(fid, cams, rc, tf).cpu())
    ctx.cube_free(aid)
    ctx.cube_free(fid)


def test_injected_h2d_failure(ctx, cube128):
    import paper_1111_6661_b300 as vrc
    v = cube128[:32, :32, :32].copy()
    sid, _ = make_streamed(ctx, v, 16)
    ctx.debug_inject("h2d", 3)
    with pytest.raises(vrc.VrcError, match="INJECTED"):
        ctx.render_mip(sid, cubegen.orbit_cameras((32, 32, 32), 1), vrc.raycfg(16, 16, 0.5))
    torch.cuda.synchronize()
    out = ctx.render_mip(sid, cubegen.orbit_cameras((32, 32, 32), 1), vrc.raycfg(16, 16, 0.5))  # recovers
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    ctx.cube_free(sid)


def test_zero_copy_matches_streamed(ctx, cube128):
    """Zero-copy variant: the brick kernels read the pinned host slots in place
    (mapped memory) instead of copying them to a device ring.  It runs the
    resident sort-last schedule, so it is bit-identical to the resident cube's
    sort-last render, and within the DVR tolerance of the streamed render (whose
    wavefronts are split into ring-sized chunks)."""
    import paper_1111_6661_b300 as vrc
    v = cube128[:64, :48, :80].copy()
    dims = (80, 48, 64)
    sid, _ = make_streamed(ctx, v, 16, ring=4)
    rid = ctx.cube_upload(v, "f32", brick=16)
    cams = cubegen.orbit_cameras(dims, 2)
    tf = cubegen.tf_dense()
    zc = vrc.raycfg(40, 32, 0.5, path="zerocopy")
    z = ctx.render_dvr(sid, cams, zc, tf).cpu()
    assert torch.equal(z, ctx.render_dvr(rid, cams, vrc.raycfg(40, 32, 0.5, path="sortlast"), tf).cpu())
    assert (z - ctx.render_dvr(sid, cams, vrc.raycfg(40, 32, 0.5), tf).cpu()).abs().max() <= 1e-4
    z = ctx.render_mip(sid, cams, zc).cpu()
    assert torch.equal(z, ctx.render_mip(sid, cams, vrc.raycfg(40, 32, 0.5)).cpu())
    with pytest.raises(vrc.VrcError, match="UNSUPPORTED"):
        ctx.render_mip(rid, cams, zc)
    ctx.cube_free(rid)
    ctx.cube_free(sid)


def test_zero_copy_aliased_slots(ctx, cube128):
    """With fewer host slots than bricks, the zero-copy path reads slot b % n."""
    import paper_1111_6661_b300 as vrc
    v = cube128[:48, :48, :48].copy()
    K = 5
    aid, _ = make_streamed(ctx, v, 16, n_host=K)
    fid, _ = make_streamed(ctx, v, 16, n_host=None, source=lambda b: b % K)
    cams = cubegen.orbit_cameras((48, 48, 48), 2)
    rc = vrc.raycfg(32, 32, 0.5, path="zerocopy")
    tf = cubegen.tf_sparse()
    assert torch.equal(ctx.render_dvr(aid, cams, rc, tf).cpu(), ctx.render_dvr(fid, cams, rc, tf).cpu())
    ctx.cube_free(aid)
    ctx.cube_free(fid)


def _tf_threshold(u0):
    t = cubegen.tf_sparse()
    t[: int(np.ceil(u0 * 255)), 3] = 0.0
    return t


@pytest.mark.parametrize("path", ["sortlast", "streamed", "zerocopy"])
def test_brick_culling_is_exact(ctx, cube128, path):
    """skip_empty on the sort-last paths culls bricks whose maximum (halo
    included) is transparent under the TF; the image is bit-identical and the
    culled bricks are neither rendered nor (streamed) copied."""
    import paper_1111_6661_b300 as vrc
    v = cube128[:64, :48, :80].copy()
    dims = (80, 48, 64)
    if path == "sortlast":
        cid = ctx.cube_upload(v, "f32", brick=16)
    else:
        cid, _ = make_streamed(ctx, v, 16, ring=4)
    p = "sortlast" if path == "sortlast" else ("zerocopy" if path == "zerocopy" else "fused")
    cams = cubegen.orbit_cameras(dims, 2) + [cubegen.ortho_z_camera(dims)]
    for tf in (cubegen.tf_sparse(), _tf_threshold(0.3), cubegen.tf_dense()):
        a = ctx.render_dvr(cid, cams, vrc.raycfg(40, 32, 0.5, path=p), tf).cpu()
        t0, c0 = ctx.last_render_bricks()
        b = ctx.render_dvr(cid, cams, vrc.raycfg(40, 32, 0.5, path=p, skip_empty=True), tf).cpu()
        t1, c1 = ctx.last_render_bricks()
        assert torch.equal(a, b)
        assert c0 == 0 and t1 + c1 == t0
        if tf[0, 3] > 0:
            assert c1 == 0          # no transparent range: nothing to cull
    assert c1 == 0
    b = ctx.render_dvr(cid, cams, vrc.raycfg(40, 32, 0.5, path=p, skip_empty=True), _tf_threshold(0.3)).cpu()
    assert ctx.last_render_bricks()[1] > 0
    # MIP never culls
    ctx.render_mip(cid, cams, vrc.raycfg(40, 32, 0.5, path=p, skip_empty=True))
    assert ctx.last_render_bricks()[1] == 0
    ctx.cube_free(cid)


def test_brick_culling_keeps_inf_halo(ctx):
    """A +inf voxel on a brick face is visible (u clamps to 1) from the
    neighbouring brick through its halo: neither brick may be culled."""
    import paper_1111_6661_b300 as vrc
    v = np.zeros((32, 32, 48), dtype=np.float32)
    v[:, :, :] = np.linspace(0.0, 1.0, 48, dtype=np.float32)[None, None, :] * 0.01
    v[0, 0, 0] = 100.0            # sets the range
    v[16, 16, 16] = np.inf        # first voxel of brick (1,1,1)
    cid = ctx.cube_upload(v, "f32", brick=16)
    tf = _tf_threshold(0.5)
    cams = [cubegen.camera("persp", (60.0, 50.0, -40.0), (24.0, 16.0, 16.0), (0, 1, 0), fovy_deg=40)]
    a = ctx.render_dvr(cid, cams, vrc.raycfg(64, 64, 0.5, path="sortlast"), tf).cpu()
    b = ctx.render_dvr(cid, cams, vrc.raycfg(64, 64, 0.5, path="sortlast", skip_empty=True), tf).cpu()
    assert torch.equal(a, b)
    assert float(a[..., 3].max()) > 0
    ctx.cube_free(cid)


def test_unfilled_streamed_cube_is_rejected(ctx, cube128):
    import paper_1111_6661_b300 as vrc
    v = cube128[:32, :32, :32].copy()
    cid = ctx.cube_create_streamed((32, 32, 32), 16, 8, 4)
    ctx.cube_put_brick(cid, 0, brick_with_halo(v, 16, 0, (2, 2, 2)))
    with pytest.raises(vrc.VrcError, match="INVAL"):
        ctx.render_mip(cid, cubegen.orbit_cameras((32, 32, 32), 1), vrc.raycfg(16, 16, 0.5))
    ctx.cube_free(cid)


def _provider(v, B):
    """Python brick provider over cube v (z, y, x) that counts its calls."""
    dims = (v.shape[2], v.shape[1], v.shape[0])
    nb = [(d + B - 1) // B for d in dims]
    calls = []

    def source(b, bx, by, bz):
        calls.append(b)
        assert b == (bz * nb[1] + by) * nb[0] + bx
        return brick_with_halo(v, B, b, nb)
    return source, calls


def _check_stats_equal(got, ref, hist_got, hist_ref):
    assert got["min"] == ref["min"] and got["max"] == ref["max"]
    assert got["n"] == ref["n"] and got["n_nonfinite"] == ref["n_nonfinite"]
    assert abs(got["mean"] - ref["mean"]) <= 1e-9 * max(abs(ref["mean"]), ref["std"])
    assert abs(got["std"] - ref["std"]) <= 1e-9 * ref["std"]
    assert np.array_equal(hist_got, hist_ref)


@pytest.mark.parametrize("n_host", [None, 3, 20])
def test_provider_cube_matches_resident_and_oracle(ctx, cube128, n_host):
    """Out-of-core cube whose bricks come from a provider (Sec. 2: a cube larger
    than memory read sub-cube by sub-cube).  With a host cache of every brick
    the provider is called once per brick; with 3 slots every render and
    statistics pass asks for bricks again.  Renders, statistics, histogram and
    median must equal those of the resident cube and the oracle."""
    import paper_1111_6661_b300 as vrc
    v = cube128[:64, :48, :80].copy()
    v[40, 10, 70] = np.nan                   # a non-finite voxel in a border brick
    dims = (80, 48, 64)
    source, calls = _provider(v, 16)
    nb_total = 5 * 3 * 4
    sid = ctx.cube_upload_streamed(dims, 16, source, n_host or nb_total, 4)
    assert sorted(calls) == list(range(nb_total))          # one scan of every brick
    rid = ctx.cube_upload(v, "f32", brick=16)
    info = ctx.cube_info(sid)
    fin = v[np.isfinite(v)]
    assert info["vmin"] == fin.min() and info["vmax"] == fin.max()
    cams = cubegen.orbit_cameras(dims, 2) + [cubegen.camera("persp", (30.2, 20.5, 31.7), (0, 0, 0), (0, 1, 0),
                                                            fovy_deg=70)]
    rc = vrc.raycfg(40, 32, 0.5)
    n0 = len(calls)
    a = ctx.render_mip(sid, cams, rc).cpu()
    assert torch.equal(a, ctx.render_mip(rid, cams, rc).cpu())
    assert (len(calls) == n0) == (n_host is None)            # cache hits only when every brick fits
    tf = cubegen.tf_dense()
    a = ctx.render_dvr(sid, cams, rc, tf).cpu().numpy().reshape(len(cams), -1, 4).astype(np.float64)
    b = ctx.render_dvr(rid, cams, rc, tf).cpu().numpy().reshape(len(cams), -1, 4)
    assert np.abs(a - b).max() <= 1e-4
    for i, cam in enumerate(cams):
        r = oracle.render(v, cam, 40, 32, 0.5, "trilinear", "dvr", tf=tf, vmin=info["vmin"], vmax=info["vmax"])
        d = np.abs(a[i] - r["out"]).max(axis=1)
        ok = (d <= 1e-4) | (r["fragile"] & np.all((a[i] >= r["lo"] - 1e-4) & (a[i] <= r["hi"] + 1e-4), axis=1))
        assert ok.all()
    # statistics and the median (Sec. 3) stream the bricks through the ring
    s, h = ctx.cube_stats(sid, 300)
    sr, hr = ctx.cube_stats(rid, 300)
    _check_stats_equal(s, sr, h, hr)
    ref = oracle.stats(v)
    _check_stats_equal(s, ref, h, oracle.histogram(v, ref["min"], ref["max"], 300))
    assert s["n_nonfinite"] == 1
    m = ctx.cube_median(sid)
    assert m == ctx.cube_median(rid) == oracle.median(v)
    ctx.cube_free(sid)
    ctx.cube_free(rid)


def test_cubegen_provider_equals_generated_cube(ctx):
    """The generator's C brick provider (no Python per brick) builds, brick by
    brick, the same cube as generating it whole: renders and statistics of the
    out-of-core cube equal those of the resident upload (ragged dims: border
    bricks take clamp-to-edge halos)."""
    import paper_1111_6661_b300 as vrc
    dims = (70, 45, 33)
    src = cubegen.BrickSource(dims, 6, 21, 16)
    sid = ctx.cube_upload_streamed(dims, 16, (src.fn, src.user), 5, 2)
    nbr = 5 * 3 * 3
    assert src.calls == nbr
    v = cubegen.generate(dims, 6, 21)
    rid = ctx.cube_upload(v, "f32", brick=16)
    cams = cubegen.orbit_cameras(dims, 2) + [cubegen.ortho_z_camera(dims)]
    rc = vrc.raycfg(48, 40, 0.5)
    assert torch.equal(ctx.render_mip(sid, cams, rc).cpu(), ctx.render_mip(rid, cams, rc).cpu())
    assert src.calls > nbr                                    # 5 host slots: bricks provided again
    s, h = ctx.cube_stats(sid, 64)
    sr, hr = ctx.cube_stats(rid, 64)
    _check_stats_equal(s, sr, h, hr)
    assert ctx.cube_median(sid) == ctx.cube_median(rid)
    ctx.cube_free(sid)
    ctx.cube_free(rid)


def test_provider_failure_is_reported(ctx, cube128):
    """A provider that fails makes the call that needed the brick fail with
    VRC_E_SOURCE: at creation no cube is made; later, the render or statistics
    call fails and the context (and the cube) stay usable."""
    import paper_1111_6661_b300 as vrc
    v = cube128[:32, :32, :48].copy()
    dims = (48, 32, 32)
    source, calls = _provider(v, 16)
    fail = {"brick": 4}

    def flaky(b, bx, by, bz):
        if b == fail["brick"]:
            raise RuntimeError("no such brick")
        return source(b, bx, by, bz)
    with pytest.raises(vrc.VrcError, match="SOURCE"):
        ctx.cube_upload_streamed(dims, 16, flaky, 12, 2)
    fail["brick"] = -1
    sid = ctx.cube_upload_streamed(dims, 16, flaky, 2, 2)       # 2 host slots for 12 bricks
    cams = cubegen.orbit_cameras(dims, 1)
    rc = vrc.raycfg(24, 24, 0.5)
    good = ctx.render_mip(sid, cams, rc).cpu()
    fail["brick"] = 7
    with pytest.raises(vrc.VrcError, match="SOURCE"):
        ctx.render_mip(sid, cams, rc)
    with pytest.raises(vrc.VrcError, match="SOURCE"):
        ctx.cube_stats(sid, 16)
    torch.cuda.synchronize()
    fail["brick"] = -1
    assert torch.equal(ctx.render_mip(sid, cams, rc).cpu(), good)
    with pytest.raises(vrc.VrcError, match="UNSUPPORTED"):
        ctx.cube_put_brick(sid, 0, brick_with_halo(v, 16, 0, (3, 2, 2)))
    with pytest.raises(vrc.VrcError, match="UNSUPPORTED"):
        ctx.render_mip(sid, cams, vrc.raycfg(24, 24, 0.5, path="zerocopy"))
    ctx.cube_free(sid)


def test_stats_of_caller_filled_streamed_cube(ctx, cube128):
    """Statistics of an out-of-core cube whose host slots the caller filled
    (vrc_cube_put_brick) equal those of the resident cube."""
    v = cube128[:48, :40, :56].copy()
    sid, _ = make_streamed(ctx, v, 16, ring=2)
    rid = ctx.cube_upload(v, "f32", brick=16)
    s, h = ctx.cube_stats(sid, 4096)
    sr, hr = ctx.cube_stats(rid, 4096)
    _check_stats_equal(s, sr, h, hr)
    assert ctx.cube_median(sid) == ctx.cube_median(rid)
    ctx.cube_free(sid)
    ctx.cube_free(rid)


def _voxels(brick_array, B):
    """Logical (B+2)^3 stored elements of a brick as read by cube_read_brick
    (the row padding dropped: resident and out-of-core cubes pad rows
    differently)."""
    R, P = B + 2, brick_array.shape[2]
    O = (P - B) // 2
    return brick_array[:, :, O - 1:O - 1 + R]


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
@pytest.mark.parametrize("n_host", [None, 3])
def test_provider_cube_bf16_fp8_matches_resident(ctx, cube128, dtype, n_host):
    """Out-of-core cube kept as bf16 / fp8 (the provider hands float32 bricks;
    each is packed on the device and its stored form kept in the host cache):
    every stored brick (bf16 bits, e4m3 codes and the brick scales behind
    them), the TF range, sort-last renders, statistics, histogram and median
    equal those of the same cube uploaded with that storage.  With 3 host slots
    bricks are provided and packed again during renders and passes."""
    import paper_1111_6661_b300 as vrc
    v = cube128[:64, :48, :80].copy()
    v[40, 10, 70] = np.nan                   # non-finite voxels in border bricks
    v[3, 47, 2] = np.inf
    dims = (80, 48, 64)
    source, calls = _provider(v, 16)
    nb_total = 5 * 3 * 4
    sid = ctx.cube_upload_streamed(dims, 16, source, n_host or nb_total, 4, storage=dtype)
    assert sorted(calls) == list(range(nb_total))
    rid = ctx.cube_upload(v, dtype, brick=16)
    si, ri = ctx.cube_info(sid), ctx.cube_info(rid)
    assert si["storage"] == dtype and (si["vmin"], si["vmax"]) == (ri["vmin"], ri["vmax"])
    for b in range(nb_total):
        assert np.array_equal(_voxels(ctx.cube_read_brick(sid, b), 16), _voxels(ctx.cube_read_brick(rid, b), 16)), b
    cams = cubegen.orbit_cameras(dims, 2) + [cubegen.ortho_z_camera(dims)]
    rc, rs = vrc.raycfg(40, 32, 0.5), vrc.raycfg(40, 32, 0.5, path="sortlast")
    assert torch.equal(ctx.render_mip(sid, cams, rc).cpu(), ctx.render_mip(rid, cams, rs).cpu())
    tf = cubegen.tf_dense()
    assert torch.equal(ctx.render_dvr(sid, cams, rc, tf).cpu(), ctx.render_dvr(rid, cams, rs, tf).cpu())
    assert ctx.last_render_path() == "sortlast"
    s, h = ctx.cube_stats(sid, 300)
    sr, hr = ctx.cube_stats(rid, 300)
    _check_stats_equal(s, sr, h, hr)
    assert s["n_nonfinite"] == 2
    assert ctx.cube_median(sid) == ctx.cube_median(rid)
    if n_host is None:
        # every brick cached: the zero-copy path reads the packed slots in place
        z = ctx.render_mip(sid, cams, vrc.raycfg(40, 32, 0.5, path="zerocopy")).cpu()
        assert torch.equal(z, ctx.render_mip(sid, cams, rc).cpu())
    ctx.cube_free(sid)
    ctx.cube_free(rid)
