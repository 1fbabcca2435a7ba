"""Brick pack + quantise (Sec. 2: the cube split into sub-cubes; the stored
types of the precision form): the stored bytes of every brick, read back
through vrc_cube_read_brick, against the oracle's rounding, bit for bit --
interior, clamp-to-edge halo and zero padding.  Shapes cover full and ragged
bricks, rows that allow 16-byte loads (nx a multiple of 4) and rows that do
not, values planted in a neighbour's halo (they must set the FP8 scale), and
non-finite voxels (the scan's second sweep)."""
import numpy as np
import pytest

import cubegen
import oracle

pytestmark = pytest.mark.gpu

ESIZE = {"f32": 4, "bf16": 2, "fp8": 1}


def e4m3_code(q: np.ndarray) -> np.ndarray:
    """Bit pattern of exact e4m3 values (|q| <= 448): sign, 4-bit exponent
    (bias 7, 0 = subnormal), 3-bit mantissa; NaN is 0x7f."""
    nan = np.isnan(q)
    q = np.where(nan, 0.0, q)
    a = np.abs(q)
    code = np.zeros(q.shape, dtype=np.uint8)
    sub = (a > 0) & (a < 2.0 ** -6)
    code[sub] = np.rint(a[sub] / 2.0 ** -9).astype(np.uint8)
    nrm = a >= 2.0 ** -6
    f, x = np.frexp(a[nrm])                 # a = f * 2^x, f in [0.5, 1)
    e = x - 1
    m = np.rint((f * 2.0 - 1.0) * 8).astype(np.int64)
    code[nrm] = (((e + 7) << 3) | m).astype(np.uint8)
    code = code | (np.signbit(q).astype(np.uint8) << 7)
    code[nan] = 0x7f
    return code


def expected_brick(v: np.ndarray, B: int, b: int, dtype: str, scales) -> np.ndarray:
    NZ, NY, NX = v.shape
    nb = [(NX + B - 1) // B, (NY + B - 1) // B, (NZ + B - 1) // B]
    bx, by, bz = b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])
    span = np.arange(-1, B + 1)
    ix = np.clip(bx * B + span, 0, NX - 1)
    iy = np.clip(by * B + span, 0, NY - 1)
    iz = np.clip(bz * B + span, 0, NZ - 1)
    blk = v[np.ix_(iz, iy, ix)]
    O = 32 // ESIZE[dtype]
    R, P = B + 2, B + 2 * O
    if dtype == "f32":
        out = np.zeros((R, R, P), dtype=np.uint32)
        codes = blk.view(np.uint32)
    elif dtype == "bf16":
        out = np.zeros((R, R, P), dtype=np.uint16)
        codes = (oracle.bf16_round(blk).view(np.uint32) >> 16).astype(np.uint16)
    else:
        out = np.zeros((R, R, P), dtype=np.uint8)
        y = (blk / np.float32(scales[b])).astype(np.float32)
        codes = e4m3_code(oracle.e4m3_round(y))
    out[:, :, O - 1:O + B + 1] = codes
    return out


def check_cube(ctx, v, B, dtype, src=None):
    dims = (v.shape[2], v.shape[1], v.shape[0])
    cid = ctx.cube_upload(v if src is None else src, dtype, brick=B)
    try:
        info = ctx.cube_info(cid)
        scales = oracle.brick_scales(v, B) if dtype == "fp8" else None
        for b in range(info["n_bricks"]):
            got = ctx.cube_read_brick(cid, b)
            want = expected_brick(v, B, b, dtype, scales)
            got = got.view(np.uint32) if dtype == "f32" else got
            if dtype == "bf16":
                # NaN payloads are not fixed by rounding: any bf16 NaN pattern matches a NaN
                nan_w = ((want & 0x7F80) == 0x7F80) & ((want & 0x7F) != 0)
                nan_g = ((got & 0x7F80) == 0x7F80) & ((got & 0x7F) != 0)
                got = np.where(nan_w & nan_g, want, got)
            bad = np.argwhere(got != want)
            assert bad.size == 0, (dims, B, dtype, b, bad[:4].tolist())
        return info
    finally:
        ctx.cube_free(cid)


@pytest.fixture(scope="module")
def ctx():
    import paper_1111_6661_b300 as vrc
    c = vrc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
@pytest.mark.parametrize("dims,B", [((96, 40, 20), 32),     # nx % 4 == 0: 16-byte loads; ragged y, z
                                    ((70, 45, 33), 16),     # nx % 4 != 0: element loads; ragged everywhere
                                    ((128, 64, 64), 64)])   # full bricks
def test_stored_bricks_bit_exact(ctx, dims, B, dtype):
    v = cubegen.generate(dims, 6, 41)
    # large magnitudes one voxel outside brick 0 (its halo) and at a far corner
    v[0, 0, min(B, dims[0] - 1)] = 900.0
    v[-1, -1, -1] = -1200.0
    check_cube(ctx, v, B, dtype)


def test_fp8_scale_counts_the_halo(ctx):
    """A brick whose largest magnitude sits in its halo takes its scale from
    it: every code of that brick then differs from an interior-only scale."""
    B = 16
    v = cubegen.generate((48, 32, 32), 4, 43)
    v[5, 5, B] = 5000.0                 # x = 16: brick 1's interior, brick 0's halo
    info = check_cube(ctx, v, B, "fp8")
    assert info["n_bricks"] == 3 * 2 * 2
    assert oracle.brick_scales(v, B)[0] == np.float32(5000.0) / np.float32(448.0)


def test_nonfinite_voxels_stored_and_skipped(ctx):
    """NaN and infinities are stored as they are (fp32), left out of the
    recorded extrema, and counted by the statistics."""
    v = cubegen.generate((64, 48, 40), 5, 44)
    v[3, 4, 5] = np.nan
    v[30, 40, 60] = np.inf
    v[39, 0, 33] = -np.inf
    info = check_cube(ctx, v, 32, "f32")
    fin = v[np.isfinite(v)]
    assert info["vmin"] == fin.min() and info["vmax"] == fin.max()
    cid = ctx.cube_upload(v, "f32", brick=32)
    try:
        s, _ = ctx.cube_stats(cid, 16)
        assert s["n_nonfinite"] == 3 and s["n"] == fin.size
        assert s["min"] == fin.min() and s["max"] == fin.max()
    finally:
        ctx.cube_free(cid)


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_nonfinite_voxels_quantised(ctx, dtype):
    """bf16 keeps NaN and infinities; e4m3 has no infinity and stores every
    non-finite voxel as NaN (0x7f), so the statistics skip them in every
    storage type."""
    v = cubegen.generate((40, 36, 20), 5, 47)
    v[3, 4, 5] = np.nan
    v[10, 20, 30] = np.inf
    v[19, 0, 33] = -np.inf
    check_cube(ctx, v, 16, dtype)
    dq = oracle.dequantize(v, dtype, 16)
    assert int(np.isnan(dq).sum()) == (1 if dtype == "bf16" else 3)
    cid = ctx.cube_upload(v, dtype, brick=16)
    try:
        s, h = ctx.cube_stats(cid, 64)
        ref = oracle.stats(dq)
        assert s["n_nonfinite"] == ref["n_nonfinite"] == 3 and s["n"] == ref["n"]
        assert s["min"] == ref["min"] and s["max"] == ref["max"]
        assert abs(s["mean"] - ref["mean"]) <= 1e-9 * max(abs(ref["mean"]), ref["std"])
        assert abs(s["std"] - ref["std"]) <= 1e-9 * ref["std"]
        assert np.array_equal(h, oracle.histogram(dq, ref["min"], ref["max"], 64))
    finally:
        ctx.cube_free(cid)


@pytest.mark.parametrize("dtype", ["f32", "fp8"])
def test_device_source_off_16_bytes(ctx, dtype):
    """A device source whose address is 4 bytes past a 16-byte boundary (a
    tensor view): rows whose length is a multiple of 4 would allow 16-byte
    loads, but the address does not, so the passes fall back to element
    loads.  Same stored bytes as from an aligned source."""
    import torch
    v = cubegen.generate((64, 40, 24), 4, 48)
    flat = torch.zeros(v.size + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(v.reshape(-1)).cuda()
    src = flat[1:].view(v.shape)
    assert src.data_ptr() % 16 == 4
    check_cube(ctx, v, 32, dtype, src=src)


def test_read_brick_errors(ctx):
    import paper_1111_6661_b300 as vrc
    v = cubegen.generate((32, 32, 32), 2, 45)
    cid = ctx.cube_upload(v, "f32", brick=16)
    try:
        with pytest.raises(vrc.VrcError):
            ctx.cube_read_brick(cid, 8)           # 2x2x2 bricks: 0..7
        with pytest.raises(vrc.VrcError):
            ctx.cube_read_brick(cid, -1)
    finally:
        ctx.cube_free(cid)
    with pytest.raises(vrc.VrcError):
        ctx.cube_read_brick(cid, 0)               # freed id
    sid = ctx.cube_create_streamed((32, 32, 32), 16, 8)
    try:
        with pytest.raises(vrc.VrcError, match="INVAL"):
            ctx.cube_read_brick(sid, 0)           # host slots not written yet
    finally:
        ctx.cube_free(sid)


def test_largest_brick_edge(ctx):
    """B = 512 (the largest brick edge): stored bricks bit-exact, and the
    macro-cell maxima (their pass needs more than 48 KB of shared memory per
    block at this edge) leave the skip_empty image bit-identical."""
    import torch

    import paper_1111_6661_b300 as vrc
    dims = (520, 24, 16)                           # 2 x 1 x 1 bricks, the second one ragged
    v = cubegen.generate(dims, 3, 46)
    check_cube(ctx, v, 512, "f32")
    cid = ctx.cube_upload(v, "f32", brick=512)
    try:
        cams = cubegen.orbit_cameras(dims, 2)
        tf = cubegen.tf_sparse()
        a = ctx.render_dvr(cid, cams, vrc.raycfg(64, 48, 0.5), tf).cpu()
        n0 = ctx.last_render_samples()
        b = ctx.render_dvr(cid, cams, vrc.raycfg(64, 48, 0.5, skip_empty=True), tf).cpu()
        n1, e1 = ctx.last_render_samples(evaluated=True)
        assert torch.equal(a, b) and n0 == n1 and e1 < n1
    finally:
        ctx.cube_free(cid)
