"""The seeded input generator: its brick provider (used for out-of-core cubes)
must give, brick by brick, exactly the cube that is generated whole, with
clamp-to-edge halos at the cube's border."""
import numpy as np
import pytest

import cubegen


@pytest.mark.parametrize("dims,B", [((40, 36, 28), 16), ((32, 32, 32), 16), ((17, 9, 5), 8)])
def test_brick_source_equals_whole_cube(dims, B):
    v = cubegen.generate(dims, 5, 7)
    src = cubegen.BrickSource(dims, 5, 7, B)
    nb = [(d + B - 1) // B for d in dims]
    for b in range(nb[0] * nb[1] * nb[2]):
        bx, by, bz = b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])
        idx = [np.clip(np.arange(o * B - 1, o * B + B + 1), 0, n - 1) for o, n in zip((bz, by, bx), v.shape)]
        assert np.array_equal(src.brick(b, nb), v[np.ix_(*idx)]), b
    assert src.calls == nb[0] * nb[1] * nb[2]
