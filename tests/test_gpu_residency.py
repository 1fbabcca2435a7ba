"""Registered cubes under an HBM budget (Abstract, Sec. 3: a shared service
keeps many users' cubes; on one GPU it holds as many resident as its memory
allows), render-copy flags and the reported render path."""
import numpy as np
import pytest
import torch

import cubegen

pytestmark = pytest.mark.gpu

MB = 1 << 20


def _cubes(n, side=256):
    return [cubegen.generate((side, side, side), 4, 300 + i) for i in range(n)]


def test_requests_wait_for_memory_and_cubes_are_evicted():
    """Three 256^3 cubes with render copies under a budget that holds one of
    them while another uploads: requests for a cube that is not resident wait
    in the queue (memory_wait_ms > 0) until an idle cube is evicted, and every
    result equals that of the same cube uploaded for good."""
    import paper_1111_6661_b300 as vrc
    vols = _cubes(3)
    ref = vrc.Context(0)
    rids = [ref.cube_upload(v, "f32", brick=128) for v in vols]
    ctx = vrc.Context(0, hbm_budget_bytes=340 * MB, n_streams=2, max_inflight=8)
    ids = [ctx.cube_register(v, "f32", brick=128) for v in vols]
    assert ctx.residency() == dict(resident=0, loads=0, evictions=0)
    assert ctx.memory()[0] == 0                       # nothing on the device yet
    dims = (256, 256, 256)
    cams = cubegen.random_cameras(dims, 6, 5)
    tf = cubegen.tf_dense()
    rc = vrc.raycfg(96, 64, 0.5)
    order = [0, 1, 2, 0, 2, 1, 1, 0]
    outs, tickets = [], []
    for k, i in enumerate(order):
        if k % 3 == 2:
            out = torch.zeros(64, dtype=torch.int64, device="cuda")
            tickets.append(("stats", i, ctx.submit("stats", ids[i], nbins=64, out=out)))
        else:
            out = torch.zeros(96 * 64 * 4, device="cuda")
            tickets.append(("dvr", i, ctx.submit("dvr", ids[i], cam=cams[k % 6], rc=rc, tf=tf, out=out)))
        outs.append(out)
    res = [ctx.poll(t, -1) for _, _, t in tickets]
    assert all(r["status"] == 0 for r in res), res
    assert max(r["memory_wait_ms"] for r in res) > 0.0
    assert any(r["cube_loaded"] for r in res)
    st = ctx.residency()
    assert st["evictions"] >= 2 and st["loads"] >= 3 and st["resident"] <= 2
    assert ctx.memory()[0] <= 340 * MB
    for k, ((kind, i, _), r, out) in enumerate(zip(tickets, res, outs)):
        if kind == "stats":
            s, h = ref.cube_stats(rids[i], 64)
            assert r["stats"] == s and np.array_equal(out.cpu().numpy().astype(np.uint64), h)
        else:
            assert r["path"] == "fused"                  # registered cubes keep their render copy
            want = ref.render_dvr(rids[i], [cams[k % 6]], rc, tf).reshape(-1)
            assert torch.equal(out, want)
    # a direct call makes a registered cube resident on the calling thread
    img = ctx.render_mip(ids[1], [cams[0]], vrc.raycfg(40, 40, 0.5))
    assert torch.equal(img, ref.render_mip(rids[1], [cams[0]], vrc.raycfg(40, 40, 0.5)))
    for i in ids:
        ctx.cube_free(i)
    ctx.close()
    ref.close()


def test_registered_cube_larger_than_budget_fails():
    import paper_1111_6661_b300 as vrc
    v = cubegen.generate((256, 256, 256), 4, 9)
    ctx = vrc.Context(0, hbm_budget_bytes=64 * MB)
    cid = ctx.cube_register(v, "f32", brick=128)
    t = ctx.submit("stats", cid, nbins=8)
    assert ctx.poll(t, -1)["status"] == -2               # VRC_E_NOMEM
    with pytest.raises(vrc.VrcError, match="NOMEM"):
        ctx.cube_stats(cid, 8)
    ctx.cube_free(cid)
    ctx.close()


def test_render_copy_flags_and_reported_path():
    """The render copy is an accelerator: AUTO drops it when the budget has no
    room (the render then takes, and reports, the global-load path), REQUIRED
    fails with VRC_E_NOMEM instead, NONE never makes it.  Every path gives the
    same image."""
    import paper_1111_6661_b300 as vrc
    v = cubegen.generate((128, 128, 128), 6, 11)
    cam = cubegen.orbit_cameras((128, 128, 128), 3)[1]
    rc = vrc.raycfg(64, 48, 0.5)
    tf = cubegen.tf_sparse()
    big = vrc.Context(0)
    a = big.cube_upload(v, "f32", brick=64)
    assert big.cube_info(a)["render_copy_bytes"] > 0
    img = big.render_dvr(a, [cam], rc, tf)
    assert big.last_render_path() == "fused"
    b = big.cube_upload(v, "f32", brick=64, render_copy="none")
    assert big.cube_info(b)["render_copy_bytes"] == 0
    assert torch.equal(big.render_dvr(b, [cam], rc, tf), img)
    assert big.last_render_path() == "fused_ldg"
    big.render_dvr(a, [cam], vrc.raycfg(64, 48, 0.5, path="sortlast"), tf)
    assert big.last_render_path() == "sortlast"
    big.render_mip(a, [cam], vrc.raycfg(64, 48, 0.5, "nearest"))
    assert big.last_render_path() == "fused_ldg"         # nearest reads the bricks
    big.close()
    # a budget that holds the bricks and the upload's staging but not the copy
    small = vrc.Context(0, hbm_budget_bytes=25 * MB)
    with pytest.raises(vrc.VrcError, match="NOMEM"):
        small.cube_upload(v, "f32", brick=64, render_copy="required")
    assert small.memory()[0] == 0                        # nothing left behind
    c = small.cube_upload(v, "f32", brick=64)            # AUTO: no room for the copy's reserve
    assert small.cube_info(c)["render_copy_bytes"] == 0
    assert torch.equal(small.render_dvr(c, [cam], rc, tf), img)
    assert small.last_render_path() == "fused_ldg"
    small.cube_free(c)
    small.close()


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_registered_bf16_fp8_load_from_packed_host_copy(dtype):
    """bf16 / fp8 registered cubes are packed once at registration; their
    packed bricks stay in page-locked host memory and every later load copies
    those: the caller's arrays are zeroed after registration and every result
    (served or direct, after evictions and reloads) still equals that of the
    same cube uploaded for good."""
    import paper_1111_6661_b300 as vrc
    vols = _cubes(3)
    ref = vrc.Context(0)
    rids = [ref.cube_upload(v, dtype, brick=128) for v in vols]
    # budgets that hold one cube's upload beside another resident cube, not all three
    budget = {"bf16": 340, "fp8": 160}[dtype] * MB
    ctx = vrc.Context(0, hbm_budget_bytes=budget, n_streams=2, max_inflight=8)
    srcs = [v.copy() for v in vols]
    ids = [ctx.cube_register(s, dtype, brick=128) for s in srcs]
    st0 = ctx.residency()
    assert st0["loads"] == 3 and st0["resident"] >= 1
    for s in srcs:
        s[...] = 0.0                                  # not read after the registration
    dims = (256, 256, 256)
    cams = cubegen.random_cameras(dims, 6, 7)
    tf = cubegen.tf_dense()
    rc = vrc.raycfg(96, 64, 0.5)
    order = [0, 1, 2, 0, 2, 1, 1, 0]
    outs, tickets = [], []
    for k, i in enumerate(order):
        if k % 3 == 2:
            out = torch.zeros(64, dtype=torch.int64, device="cuda")
            tickets.append(("stats", i, ctx.submit("stats", ids[i], nbins=64, out=out)))
        else:
            out = torch.zeros(96 * 64 * 4, device="cuda")
            tickets.append(("dvr", i, ctx.submit("dvr", ids[i], cam=cams[k % 6], rc=rc, tf=tf, out=out)))
        outs.append(out)
    res = [ctx.poll(t, -1) for _, _, t in tickets]
    assert all(r["status"] == 0 for r in res), res
    st = ctx.residency()
    assert st["loads"] > 3 and st["evictions"] >= 2
    for k, ((kind, i, _), r, out) in enumerate(zip(tickets, res, outs)):
        if kind == "stats":
            s, h = ref.cube_stats(rids[i], 64)
            assert r["stats"] == s and np.array_equal(out.cpu().numpy().astype(np.uint64), h)
        else:
            assert r["path"] == "fused"
            assert torch.equal(out, ref.render_dvr(rids[i], [cams[k % 6]], rc, tf).reshape(-1))
    img = ctx.render_mip(ids[2], [cams[1]], vrc.raycfg(40, 40, 0.5))
    assert torch.equal(img, ref.render_mip(rids[2], [cams[1]], vrc.raycfg(40, 40, 0.5)))
    assert ctx.cube_median(ids[0]) == ref.cube_median(rids[0])
    for i in ids:
        ctx.cube_free(i)
    ctx.close()
    ref.close()
