"""Pins of the oracle's ray casting (sub-cube rendering and gathering of
partial images, Sec. 2 / Table 1) against closed forms, brute force and
invariants."""
import math

import numpy as np
import pytest

import cubegen
import oracle
import naive

F32MAX = float(np.finfo(np.float32).max)


def test_axis_aligned_nearest_mip_is_column_max(cube128):
    cam = cubegen.ortho_z_camera((128, 128, 128))
    r = oracle.render(cube128, cam, 256, 256, 1.0, "nearest", "mip")
    col = cube128.max(axis=0).astype(np.float64)
    img = r["out"].reshape(256, 256)
    # pixel (u, v) samples the column (u // 2, v // 2)
    assert np.array_equal(img, np.repeat(np.repeat(col, 2, 0), 2, 1))
    assert np.all(r["nsamp"] == 128)


def test_axis_aligned_native_resolution_mip_all_modes(cube128):
    v = cube128[:40, :24, :32]
    cam = cubegen.ortho_z_camera((32, 24, 40))
    col = v.max(axis=0).astype(np.float64)
    for sampling in ("nearest", "trilinear"):
        r = oracle.render(v, cam, 32, 24, 1.0, sampling, "mip")
        # rays through voxel centres with step 1 hit voxel centres exactly
        assert np.array_equal(r["out"].reshape(24, 32), col), sampling


def test_ortho_ray_setup_closed_form():
    dims = (128, 128, 128)
    cam = cubegen.ortho_z_camera(dims)
    for px, py in [(0, 0), (255, 0), (17, 200), (255, 255)]:
        hit, o, d, t = oracle.ray(cam, 256, 256, px, py, dims)
        assert hit
        assert list(o) == [(px + 0.5) / 2, (py + 0.5) / 2, 0.0]
        assert list(d) == [0.0, 0.0, 1.0] and list(t) == [0.0, 128.0]


def test_perspective_rays_match_binary64_geometry():
    dims = (64, 48, 80)
    cams = cubegen.orbit_cameras(dims, 5) + cubegen.random_cameras(dims, 3, seed=9)
    W, H = 40, 30
    for cam in cams:
        for px, py in [(0, 0), (39, 0), (20, 15), (3, 29)]:
            hit, o, d, t = oracle.ray(cam, W, H, px, py, dims)
            o64, d64 = naive.camera_rays(cam, W, H, px, py)
            assert np.allclose(d, d64, atol=2e-6) and np.allclose(o, o64, atol=1e-3)
            tt = naive.slab(o64, d64, dims)
            assert hit == (tt is not None)
            if hit:
                assert abs(t[0] - tt[0]) < 1e-3 and abs(t[1] - tt[1]) < 1e-3


def test_perspective_symmetry():
    # looking straight down -z at the centre: pixel (px, py) and its mirror image
    # through the image centre have mirrored directions
    dims = (32, 32, 32)
    cam = cubegen.camera("persp", (16, 16, 100), (16, 16, 16), (0, 1, 0), fovy_deg=30)
    W = H = 16
    for px, py in [(0, 0), (3, 11), (7, 8)]:
        _, _, d1, _ = oracle.ray(cam, W, H, px, py, dims)
        _, _, d2, _ = oracle.ray(cam, W, H, W - 1 - px, H - 1 - py, dims)
        assert abs(d1[0] + d2[0]) < 1e-6 and abs(d1[1] + d2[1]) < 1e-6 and abs(d1[2] - d2[2]) < 1e-6
        assert d1[2] < 0


def test_single_peak_renders_peak():
    v = np.zeros((9, 8, 7), np.float32)
    v[4, 3, 5] = 17.5
    cam = cubegen.ortho_z_camera((7, 8, 9))
    for sampling in ("nearest", "trilinear"):
        r = oracle.render(v, cam, 7, 8, 1.0, sampling, "mip")
        img = r["out"].reshape(8, 7)
        assert img[3, 5] == 17.5
        assert np.count_nonzero(img) == 1
    # perspective ray aimed through the voxel centre
    cam = cubegen.camera("persp", (5.5, 3.5, -40), (5.5, 3.5, 4.5), (0, 1, 0), fovy_deg=20)
    # entry at z = 0, step 1: sample 4 sits at z = 4.5, the voxel centre
    r = oracle.render(v, cam, 9, 9, 1.0, "trilinear", "mip", pixels=[4 * 9 + 4])
    assert abs(r["out"][0] - 17.5) < 17.5 * 1e-5
    # step 0.25 straddles the centre at 4.375 / 4.625: weight 7/8 on the peak
    r = oracle.render(v, cam, 9, 9, 0.25, "trilinear", "mip", pixels=[4 * 9 + 4])
    assert abs(r["out"][0] - 17.5 * 0.875) < 17.5 * 1e-5


@pytest.mark.parametrize("alpha", [0.05, 0.3, 0.9])
def test_uniform_alpha_closed_form(alpha):
    v = np.full((16, 4, 4), 1.0, np.float32)
    tf = cubegen.tf_constant((0.2, 0.5, 1.0), alpha)
    cam = cubegen.ortho_z_camera((4, 4, 16))
    r = oracle.render(v, cam, 4, 4, 1.0, "trilinear", "dvr", tf=tf, vmin=0, vmax=2, term=2.0)
    n = 16
    A = 1 - (1 - np.float64(np.float32(alpha))) ** n
    c = np.array([0.2, 0.5, 1.0], np.float32).astype(np.float64)
    assert np.allclose(r["out"][:, 3], A, rtol=0, atol=1e-14)
    assert np.allclose(r["out"][:, :3], c[None, :] * A, rtol=0, atol=1e-14)
    assert np.all(r["nsamp"] == n)


@pytest.mark.parametrize("alpha,step", [(0.05, 0.5), (0.3, 0.25), (0.6, 1.0)])
def test_opacity_correction_closed_form(alpha, step):
    # a sample's opacity is 1-(1-a)^step: n samples at spacing `step` through a
    # constant cube absorb exactly as n*step unit-spaced samples would
    v = np.full((16, 4, 4), 1.0, np.float32)
    tf = cubegen.tf_constant((0.2, 0.5, 1.0), alpha)
    cam = cubegen.ortho_z_camera((4, 4, 16))
    r = oracle.render(v, cam, 4, 4, step, "trilinear", "dvr", tf=tf, vmin=0, vmax=2, term=2.0,
                      opacity_correction=True)
    n = int(r["nsamp"][0])
    assert np.all(r["nsamp"] == n) and n == int(round(16 / step))
    a = np.float64(np.float32(alpha))
    A = 1 - (1 - a) ** (step * n)
    assert np.allclose(r["out"][:, 3], A, rtol=0, atol=1e-12)
    assert np.allclose(r["out"][:, :3], np.array([0.2, 0.5, 1.0], np.float32).astype(np.float64) * A, atol=1e-12)
    # without the correction the same samples absorb more (step < 1) or the same (step = 1)
    r0 = oracle.render(v, cam, 4, 4, step, "trilinear", "dvr", tf=tf, vmin=0, vmax=2, term=2.0)
    assert np.allclose(r0["out"][:, 3], 1 - (1 - a) ** n, atol=1e-12)


@pytest.mark.parametrize("alpha", [0.01, 0.05, 0.3])
def test_termination_index_closed_form(alpha):
    a = float(np.float32(alpha))
    nstar = math.ceil(math.log(0.01) / math.log(1 - a))
    v = np.full((nstar + 40, 2, 2), 1.0, np.float32)
    tf = cubegen.tf_constant((1, 1, 1), alpha)
    cam = cubegen.ortho_z_camera((2, 2, v.shape[0]))
    r = oracle.render(v, cam, 2, 2, 1.0, "nearest", "dvr", tf=tf, vmin=0, vmax=2, term=0.99)
    assert np.all(r["nsamp"] == nstar)
    assert np.allclose(r["out"][:, 3], 1 - (1 - a) ** nstar, atol=1e-14)


def _tiny_cases():
    cases = []
    for seed, dims in [(1, (2, 2, 2)), (2, (3, 4, 5)), (3, (8, 8, 8)), (4, (16, 9, 12))]:
        rng = np.random.default_rng(seed)
        v = rng.standard_normal(dims[::-1]).astype(np.float32)
        cams = [cubegen.ortho_z_camera(dims)] + cubegen.random_cameras(dims, 2, seed)
        cases.append((v, dims, cams))
    return cases


@pytest.mark.parametrize("case", range(4))
def test_brute_force_tiny_cubes(case):
    v, dims, cams = _tiny_cases()[case]
    W, H = 12, 10
    tf = cubegen.tf_random(case)
    vmin, vmax = float(v.min()), float(v.max())
    for cam in cams:
        for sampling in ("nearest", "trilinear"):
            for mode in ("mip", "dvr"):
                r = oracle.render(v, cam, W, H, 0.37, sampling, mode, tf=tf, vmin=vmin, vmax=vmax, term=2.0)
                for p in range(W * H):
                    ref, n = naive.render_pixel(v, cam, W, H, p % W, p // W, 0.37, sampling, mode, tf, vmin, vmax,
                                                term=2.0)
                    if n != r["nsamp"][p]:
                        continue  # binary64 geometry vs binary32 lattice: grazing ray
                    if sampling == "nearest":
                        # a binary64 position may fall on the other side of a voxel face
                        continue
                    got = r["out"][p]
                    assert np.allclose(got, ref, rtol=1e-4, atol=1e-4), (cam, sampling, mode, p)


def test_brute_force_exact_lattice_ortho():
    # orthographic, step 1 through voxel centres: binary32 and binary64 geometry
    # coincide, so the brute force must agree to rounding, including nearest
    rng = np.random.default_rng(8)
    dims = (6, 5, 7)
    v = rng.standard_normal(dims[::-1]).astype(np.float32)
    cam = cubegen.ortho_z_camera(dims)
    tf = cubegen.tf_random(3)
    vmin, vmax = float(v.min()), float(v.max())
    for sampling in ("nearest", "trilinear"):
        for mode in ("mip", "dvr"):
            r = oracle.render(v, cam, 6, 5, 1.0, sampling, mode, tf=tf, vmin=vmin, vmax=vmax, term=0.6)
            for p in range(30):
                ref, n = naive.render_pixel(v, cam, 6, 5, p % 6, p // 6, 1.0, sampling, mode, tf, vmin, vmax,
                                            term=0.6)
                assert n == r["nsamp"][p]
                assert np.allclose(r["out"][p], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("B", [2, 3, 5, 8])
def test_bricked_equals_unbricked(B, cube128):
    v = cube128[:20, :17, :23]
    dims = (23, 17, 20)
    cams = [cubegen.ortho_z_camera(dims)] + cubegen.orbit_cameras(dims, 3) + cubegen.random_cameras(dims, 2, B)
    # a camera inside the cube
    cams.append(cubegen.camera("persp", (11.3, 8.2, 9.7), (0, 0, 0), (0, 1, 0), fovy_deg=60))
    tf = cubegen.tf_dense()
    vmin, vmax = float(v.min()), float(v.max())
    W, H = 24, 18
    for cam in cams:
        for sampling in ("nearest", "trilinear"):
            a = oracle.render(v, cam, W, H, 0.5, sampling, "mip")
            b = oracle.render(v, cam, W, H, 0.5, sampling, "mip", brick=B)
            assert np.array_equal(a["out"], b["out"])
            a = oracle.render(v, cam, W, H, 0.5, sampling, "dvr", tf=tf, vmin=vmin, vmax=vmax)
            b = oracle.render(v, cam, W, H, 0.5, sampling, "dvr", tf=tf, vmin=vmin, vmax=vmax, brick=B)
            assert np.max(np.abs(a["out"] - b["out"])) <= 1e-12
            assert np.array_equal(a["nsamp"], b["nsamp"])


def test_empty_ray_and_background():
    v = np.ones((4, 4, 4), np.float32)
    cam = cubegen.camera("persp", (2, 2, 50), (200, 2, 50), (0, 1, 0), fovy_deg=10)  # looks away
    r = oracle.render(v, cam, 4, 4, 0.5, "trilinear", "mip")
    assert np.all(r["out"] == -F32MAX) and np.all(r["nsamp"] == 0)
    r = oracle.render(v, cam, 4, 4, 0.5, "trilinear", "dvr", tf=cubegen.tf_dense(), vmin=0, vmax=1)
    assert np.all(r["out"] == 0)


def test_nan_voxels():
    v = np.ones((4, 4, 4), np.float32)
    v[:, 1, 1] = np.nan
    cam = cubegen.ortho_z_camera((4, 4, 4))
    r = oracle.render(v, cam, 4, 4, 1.0, "nearest", "mip")
    img = r["out"].reshape(4, 4)
    assert img[1, 1] == -F32MAX and img[0, 0] == 1.0
    tf = cubegen.tf_constant((1, 1, 1), 0.5)
    r = oracle.render(v, cam, 4, 4, 1.0, "nearest", "dvr", tf=tf, vmin=0, vmax=2, term=2)
    assert np.all(r["out"][5] == 0) and r["out"][0, 3] > 0


def test_composite_over_properties():
    rng = np.random.default_rng(2)
    def img():
        a = rng.uniform(0, 1, (50, 1))
        return np.concatenate([rng.uniform(0, 1, (50, 3)) * a, a], axis=1)
    f, m, b = img(), img(), img()
    left = oracle.composite(oracle.composite(f, m), b)
    right = oracle.composite(f, oracle.composite(m, b))
    assert np.allclose(left, right, atol=1e-14)
    zero = np.zeros_like(f)
    assert np.array_equal(oracle.composite(zero, b), b)
    assert np.array_equal(oracle.composite(f, zero), f)
    x, y = rng.standard_normal(10), rng.standard_normal(10)
    assert np.array_equal(oracle.composite(x, y, "mip"), np.maximum(x, y))


def test_composite_over_values():
    """Sort-last gathering of partial images (Sec. 2) by the premultiplied
    "over" operator, pinned by value: out = front + (1 - front.A) * back on
    every channel, alpha included.  Dyadic inputs make every product and sum
    exact in binary64, so the expected values are exact."""
    # front colour c=(1, 0.5, 0.25) at alpha a=0.5, back colour c'=(0.5, 1, 0.75) at alpha b=0.25
    a, b = 0.5, 0.25
    front = np.array([[1.0 * a, 0.5 * a, 0.25 * a, a]])
    back = np.array([[0.5 * b, 1.0 * b, 0.75 * b, b]])
    want = np.array([[0.5 + 0.5 * 0.125, 0.25 + 0.5 * 0.25, 0.125 + 0.5 * 0.1875, 0.5 + 0.5 * 0.25]])
    assert np.array_equal(oracle.composite(front, back), want)
    # the back layer shows through in proportion to the front's transparency,
    # not to the back's own alpha: with an opaque back layer the result's
    # alpha is 1 whatever the front
    front2 = np.array([[0.0, 0.0, 0.375, 0.375]])
    back2 = np.array([[0.25, 0.5, 0.125, 1.0]])
    assert np.array_equal(oracle.composite(front2, back2), np.array([[0.15625, 0.3125, 0.453125, 1.0]]))
    # an opaque front hides the back completely
    opaque = np.array([[0.75, 0.5, 0.25, 1.0]])
    assert np.array_equal(oracle.composite(opaque, back2), opaque)
    # the operator is not commutative: swapping the layers changes the colour
    assert not np.array_equal(oracle.composite(back, front), oracle.composite(front, back))
    # a chain of n layers of uniform alpha a has total alpha 1 - (1 - a)^n
    layer = np.array([[0.25, 0.25, 0.25, 0.25]])
    acc = np.zeros((1, 4))
    for n in range(1, 6):
        acc = oracle.composite(acc, layer)
        assert acc[0, 3] == 1 - 0.75 ** n


def test_composite_max_values():
    """MIP partial images combine by maximum; -FLT_MAX (a ray that missed the
    brick) is the identity, and ties keep the common value."""
    f32max = float(np.finfo(np.float32).max)
    front = np.array([1.5, -f32max, 2.0, -3.0, 7.25])
    back = np.array([0.5, 4.0, 2.0, -f32max, 7.5])
    assert np.array_equal(oracle.composite(front, back, "mip"), np.array([1.5, 4.0, 2.0, -3.0, 7.5]))
    assert np.array_equal(oracle.composite(back, front, "mip"), np.array([1.5, 4.0, 2.0, -3.0, 7.5]))


def test_dvr_fragile_window_brackets_result():
    v = cubegen.generate((24, 24, 24), 3, 5)
    cam = cubegen.orbit_cameras((24, 24, 24), 4)[1]
    tf = cubegen.tf_dense()
    r = oracle.render(v, cam, 20, 20, 0.5, "trilinear", "dvr", tf=tf, vmin=float(v.min()), vmax=float(v.max()))
    assert np.all(r["lo"] <= r["out"] + 1e-15) and np.all(r["out"] <= r["hi"] + 1e-15)
    assert np.all((r["lo"] == r["hi"]).all(axis=1) | r["fragile"])


def test_fp8_bricked_render_uses_brick_copies(cube128):
    v = cube128[:16, :16, :16]
    cam = cubegen.orbit_cameras((16, 16, 16), 2)[0]
    s = oracle.brick_scales(v, 8)
    a = oracle.render(v, cam, 16, 16, 0.5, "trilinear", "mip", dtype="fp8", brick=8, scales=s)
    b = oracle.render(v, cam, 16, 16, 0.5, "trilinear", "mip")
    hit = a["nsamp"] > 0
    # fp8 storage error is bounded by the E4M3 spacing (2^-4 relative) of the values
    assert np.all(np.abs(a["out"][hit] - b["out"][hit]) <= 2 ** -4 * np.abs(v).max() + 1e-6)
    # with bf16 storage the bricked and unbricked renders agree exactly (per-voxel rounding)
    c = oracle.render(v, cam, 16, 16, 0.5, "trilinear", "mip", dtype="bf16", brick=8)
    d = oracle.render(oracle.dequantize(v, "bf16"), cam, 16, 16, 0.5, "trilinear", "mip")
    assert np.array_equal(c["out"], d["out"])
