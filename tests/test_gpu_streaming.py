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
