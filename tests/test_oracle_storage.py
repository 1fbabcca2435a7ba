"""Pins of the oracle's storage roundings (BF16 and FP8 E4M3 with a per-brick
scale) against torch's CPU conversions and closed forms."""
import numpy as np
import torch

import oracle


def _probe_values():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(20000) * 10, rng.standard_normal(2000) * 1e-38,
                        rng.uniform(-500, 500, 5000), [0.0, 1.0, 1.5, -2.75, 3.0e38]])
    return x.astype(np.float32)


def test_bf16_matches_torch_rne():
    x = _probe_values()
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(oracle.bf16_round(x), ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 lies half-way between 1 and 1 + 2^-7: even mantissa is 1
    x = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8], np.float32)
    assert list(oracle.bf16_round(x)) == [1.0, 1 + 2 ** -6]


def test_e4m3_matches_torch_in_range():
    x = _probe_values()
    x = x[np.abs(x) < 464]
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).float().numpy().astype(np.float64)
    got = oracle.e4m3_round(x)
    assert np.array_equal(got, ref)


def test_e4m3_saturates_and_closed_forms():
    x = np.array([448, 460, 500, 1e6, -1e6, 2 ** -9, 2 ** -10, 1.5 * 2 ** -9, 240, 232], np.float32)
    got = oracle.e4m3_round(x)
    assert list(got) == [448, 448, 448, 448, -448, 2 ** -9, 0, 2 ** -8, 240, 224]
    # every finite E4M3 value is a fixed point
    codes = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).float().numpy()
    codes = codes[np.isfinite(codes)]
    assert np.array_equal(oracle.e4m3_round(codes), codes.astype(np.float64))


def test_e4m3_has_no_infinity():
    """E4M3 (finite-only) has NaN as its one non-finite value: NaN and +-inf
    round to NaN, while finite overflow saturates to +-448.  A stored cube
    therefore keeps its non-finite voxels non-finite, and they do not set the
    brick scale."""
    got = oracle.e4m3_round(np.array([np.nan, np.inf, -np.inf, 3.0e38, -3.0e38], np.float32))
    assert np.isnan(got[:3]).all() and list(got[3:]) == [448.0, -448.0]
    v = np.full((4, 4, 4), 2.0, np.float32)
    v[0, 0, 0], v[1, 2, 3], v[3, 3, 3] = np.inf, -np.inf, np.nan
    s = oracle.brick_scales(v, 4)
    assert s[0] == np.float32(2.0) / np.float32(448.0)
    d = oracle.dequantize(v, "fp8", 4, s)
    assert np.isnan(d[0, 0, 0]) and np.isnan(d[1, 2, 3]) and np.isnan(d[3, 3, 3])
    assert np.all(d[np.isfinite(v)] == 2.0)
    st = oracle.stats(d)
    assert st["n_nonfinite"] == 3 and st["n"] == 61 and st["mean"] == 2.0


def test_fp8_brick_scale_and_dequant():
    rng = np.random.default_rng(5)
    v = (rng.standard_normal((12, 10, 9)) * 7).astype(np.float32)
    B = 4
    s = oracle.brick_scales(v, B)
    assert s.size == 3 * 3 * 3
    # the brick whose stored region (with halo) holds the absolute maximum maps it
    # to exactly +-448 * scale
    k, j, i = np.unravel_index(np.argmax(np.abs(v)), v.shape)
    d = oracle.dequantize(v, "fp8", B, s)
    b = ((k // B) * 3 + (j // B)) * 3 + (i // B)
    assert np.float32(np.abs(v).max()) / s[b] == np.float32(448) or abs(np.abs(v).max() / s[b] - 448) < 1e-4
    # dequantised values: e4m3(x / s) * s in binary32, errors bounded by the spacing
    rel = np.abs(d - v) / np.maximum(np.abs(v), 1e-30)
    small = np.abs(v) < 1e-2
    assert np.all(rel[~small] <= 2 ** -4 + 1e-7)


def test_bf16_dequant_is_per_voxel():
    rng = np.random.default_rng(6)
    v = rng.standard_normal((5, 6, 7)).astype(np.float32)
    d = oracle.dequantize(v, "bf16", 4)
    assert np.array_equal(d, torch.from_numpy(v).to(torch.bfloat16).float().numpy())


def test_fp8_scale_counts_the_halo():
    """The per-brick FP8 scale is absmax/448 over everything the brick stores,
    its one-voxel halo included: a magnitude that sits just outside brick 0
    (in the neighbouring brick's interior, within brick 0's halo) sets brick
    0's scale, while a brick that neither holds it nor has it in its halo
    keeps its own interior maximum."""
    B = 16
    v = np.full((32, 32, 48), 1.0, np.float32)
    v[5, 5, B] = 5000.0                 # x = 16: brick 1's interior, brick 0's halo
    s = oracle.brick_scales(v, B)
    assert s.size == 3 * 2 * 2
    assert s[0] == np.float32(5000.0) / np.float32(448.0)   # halo voxel
    assert s[1] == np.float32(5000.0) / np.float32(448.0)   # interior voxel
    assert s[2] == np.float32(1.0) / np.float32(448.0)      # x in [32, 48): neither
    # a brick whose scale came from its halo codes its own voxels on that scale
    d = oracle.dequantize(v, "fp8", B, s)
    q = np.float32(oracle.e4m3_round(np.array([np.float32(1.0) / s[0]], np.float32))[0])
    assert d[0, 0, 0] == np.float32(q * s[0])
