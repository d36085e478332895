"""Pins of the out-of-core oracle: the blocks partition the first axis into
balanced, disjoint, covering ranges; a relative tolerance uses max|u| of the
whole field; the side-by-side reconstruction keeps the L-infinity bound at
every node and one block reproduces the in-core pipeline."""
import math

import numpy as np
import pytest

from oracle import ooc, pipeline


@pytest.mark.parametrize("n0,nb", [(1, 1), (10, 3), (65, 4), (513, 7), (100, 100)])
def test_blocks_partition_the_first_axis(n0, nb):
    r = ooc.block_ranges(n0, nb)
    assert len(r) == nb and r[0][0] == 0 and r[-1][1] == n0
    assert all(a < b for a, b in r) and all(r[i][1] == r[i + 1][0] for i in range(nb - 1))
    sizes = [b - a for a, b in r]
    assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        ooc.block_ranges(n0, n0 + 1)


@pytest.mark.parametrize("shape,nb", [((40, 17, 9), 3), ((65, 33), 4), ((17,), 2)])
def test_blocks_keep_the_bound_everywhere(shape, nb):
    rng = np.random.default_rng(nb)
    u = rng.standard_normal(shape).cumsum(axis=0)
    blocks, tol_abs = ooc.compress(u, 1e-2, nb, relative=True)
    assert tol_abs == 1e-2 * np.max(np.abs(u))
    out = ooc.decompress(blocks)
    assert out.shape == u.shape
    assert np.max(np.abs(out - u)) <= tol_abs
    # one block is the in-core pipeline
    one, t1 = ooc.compress(u, tol_abs, 1)
    c = pipeline.compress(u, tol_abs, math.inf, relative=False)
    assert np.array_equal(one[0]["symbols"], c["symbols"]) and t1 == tol_abs
