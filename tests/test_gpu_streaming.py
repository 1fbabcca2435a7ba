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
