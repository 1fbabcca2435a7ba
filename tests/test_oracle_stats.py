"""Pins of the oracle's statistics (min/max and histogram: Abstract; std and
median: Sec. 3) against closed forms and library routines."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle


def test_constant_cube_closed_form():
    v = np.full((5, 6, 7), 3.25, dtype=np.float32)
    s = oracle.stats(v)
    assert s["min"] == s["max"] == 3.25
    assert s["mean"] == 3.25 and s["std"] == 0.0
    assert s["n"] == v.size and s["n_nonfinite"] == 0


@pytest.mark.parametrize("n", [1, 2, 17, 4096, 2 ** 21])
def test_linear_ramp_closed_form(n):
    v = np.arange(n, dtype=np.float32)
    s = oracle.stats(v)
    assert s["mean"] == (n - 1) / 2
    var = (n * n - 1) / 12
    assert abs(s["std"] ** 2 - var) <= 1e-12 * max(var, 1)
    assert s["min"] == 0 and s["max"] == n - 1


def test_random_vs_exact_library_sum():
    rng = np.random.default_rng(7)
    v = (rng.standard_normal(100_003) * 3 + 1e3).astype(np.float32)
    s = oracle.stats(v)
    x = v.astype(np.float64)
    mean = math.fsum(x) / x.size  # correctly rounded sum
    var = math.fsum((x - mean) ** 2) / x.size
    assert abs(s["mean"] - mean) <= 1e-15 * abs(mean)
    assert abs(s["std"] - math.sqrt(var)) <= 1e-12 * math.sqrt(var)
    assert s["min"] == x.min() and s["max"] == x.max()


def test_nonfinite_skipped_and_counted():
    v = np.array([1, np.nan, 2, np.inf, -np.inf, 3], dtype=np.float32)
    s = oracle.stats(v)
    assert (s["n"], s["n_nonfinite"]) == (3, 3)
    assert s["mean"] == 2 and s["min"] == 1 and s["max"] == 3
    assert abs(s["std"] - math.sqrt(2 / 3)) < 1e-15


def test_histogram_ramp_exact_counts():
    # values 0..256 over [0, 256] with 256 bins: scale is exactly 1, bin(i) = i and
    # the maximum lands in the last bin
    v = np.arange(257, dtype=np.float32)
    h = oracle.histogram(v, 0, 256, 256)
    exp = np.ones(256, dtype=np.uint64)
    exp[-1] = 2
    assert np.array_equal(h, exp)


@pytest.mark.parametrize("nbins", [1, 7, 256, 4096])
def test_histogram_matches_exact_rational_bins(nbins):
    rng = np.random.default_rng(nbins)
    v = rng.standard_normal(20_000).astype(np.float32)
    vmin, vmax = float(v.min()), float(v.max())
    h = oracle.histogram(v, vmin, vmax, nbins)
    assert int(h.sum()) == v.size
    # exact bin of each value in rational arithmetic; the binary32 formula may
    # only differ from it next to a bin edge
    lo, span = Fraction(vmin), Fraction(vmax) - Fraction(vmin)
    exact = np.zeros(nbins, dtype=np.int64)
    near_edge = 0
    for x in v.tolist():
        t = (Fraction(x) - lo) * nbins / span
        b = min(int(t), nbins - 1)
        exact[b] += 1
        if abs(t - round(t)) < Fraction(1, 10 ** 5) * max(1, nbins):
            near_edge += 1
    assert np.abs(exact - h.astype(np.int64)).sum() <= 2 * near_edge


def test_histogram_degenerate_range_and_nonfinite():
    v = np.array([2, 2, np.nan, 2], dtype=np.float32)
    h = oracle.histogram(v, 2, 2, 16)
    assert h[0] == 3 and h.sum() == 3


def test_histogram_sum_is_n_on_generated_cube(cube128):
    s = oracle.stats(cube128)
    h = oracle.histogram(cube128, s["min"], s["max"], 256)
    assert int(h.sum()) == cube128.size
    assert h[0] >= 1 and h[-1] >= 1  # min lands in bin 0, max in the last bin


@pytest.mark.parametrize("n", [1, 2, 3, 10, 1001])
def test_median_is_lower_order_statistic(n):
    rng = np.random.default_rng(n)
    v = rng.standard_normal(n).astype(np.float32)
    assert oracle.median(v) == np.sort(v)[(n - 1) // 2]
    w = np.concatenate([v, np.array([np.nan, np.inf], np.float32)])
    assert oracle.median(w) == np.sort(v)[(n - 1) // 2]


def test_generated_cube_sanity(cube128):
    # noise-only cube: mean ~ 0, std ~ 1 (statistical sanity, not parity)
    import cubegen
    v = cubegen.generate((64, 64, 64), 0, 11)
    s = oracle.stats(v)
    assert abs(s["mean"]) < 5 / math.sqrt(v.size) and abs(s["std"] - 1) < 0.01
    assert not np.any(cube128 == 0)   # no zeros, hence no -0.0 ambiguity in min/max
