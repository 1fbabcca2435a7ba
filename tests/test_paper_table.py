"""Reading of the paper's Table 1 (Sec. 2) used for the workload sizes: voxels
are 4-byte values and "GB" is 2^30 bytes; the 2.5 teravoxel/s claim is the
largest cube times its C2050 frame rate."""
import os

import numpy as np

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table1_fps.txt")


def test_table1_sizes_are_four_byte_voxels_in_gib():
    rows = np.loadtxt(GOLD)
    for nx, ny, nz, gb, _, _ in rows:
        assert abs(nx * ny * nz * 4 / 2 ** 30 - gb) <= 0.6   # 25.48 GiB is printed as 26


def test_peak_voxel_rate_claim():
    rows = np.loadtxt(GOLD)
    rate = max(nx * ny * nz * fps for nx, ny, nz, _, _, fps in rows)
    assert abs(rate / 2 ** 40 - 2.5) < 0.02   # "2.5 teravoxel" with tera = 2^40
