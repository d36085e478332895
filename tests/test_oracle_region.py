"""Pins of the region-adaptive bound oracle: brute force over the exact
linear map from coefficient errors to the reconstruction (every column a
recomposition of a unit vector) shows that the widths keep the worst-case
error inside each box within its tolerance and within the background
tolerance everywhere; the operator norms and tails against the uniform
bound's K_l; no region reduces to the uniform widths; round trips."""
import math

import numpy as np
import pytest

from oracle import bounds, grid, multilevel, region


def _error_map(shape):
    """R[p, i]: reconstruction at p of a unit error in coefficient i."""
    N = int(np.prod(shape))
    R = np.empty((N, N))
    for i in range(N):
        e = np.zeros(N)
        e[i] = 1.0
        R[:, i] = multilevel.recompose(e.reshape(shape)).reshape(-1)
    return R


CASES = [
    ((65,), 1.0, [((20,), (30,), 1e-2), ((50,), (52,), 1e-3)]),
    ((17, 17), 1.0, [((4, 5), (8, 9), 1e-2), ((12, 0), (16, 3), 1e-3)]),
    ((9, 9, 9), 1.0, [((2, 2, 2), (5, 4, 6), 1e-3)]),
    ((33, 1, 9), 2.0, [((10, 0, 3), (12, 0, 5), 1e-2)]),
]


@pytest.mark.parametrize("shape,tol,regions", CASES)
def test_worst_case_error_within_every_tolerance(shape, tol, regions):
    w = region.node_widths(shape, tol, regions)
    worst = (np.abs(_error_map(shape)) @ (w.reshape(-1) / 2.0)).reshape(shape)
    tmap = region.tolerance_map(shape, tol, regions)
    assert np.all(worst <= tmap * (1 + 1e-12)), np.max(worst / tmap)
    # not vacuous: inside the tightest box the worst case uses a fair share
    # of its tolerance (looser boxes near it inherit its widths on small grids)
    lo, hi, tr = min(regions, key=lambda r: r[2])
    sl = tuple(slice(a, b + 1) for a, b in zip(lo, hi))
    assert np.max(worst[sl]) > 0.05 * tr


@pytest.mark.parametrize("shape,box", [((1025,), ((500,), (520,))), ((257, 257), ((100, 100), (120, 120)))])
def test_tight_widths_stay_near_the_box(shape, box):
    """On grids large against the dilation, most nodes keep the background
    width (on small grids the coarse levels' dilations cover everything)."""
    regions = [(box[0], box[1], 1e-3)]
    pl = region.plan(shape, 1.0, regions)
    w = region.node_widths(shape, 1.0, regions)
    assert np.mean(w == pl["w_bg"]) > 0.85
    assert pl["k"][0] == math.ceil(-math.log2(1e-3 - pl["far"]))


@pytest.mark.parametrize("shape", [(33,), (17, 9), (9, 10, 11), (600, 3)])
def test_axis_norms_and_tails(shape):
    h = grid.hierarchy(shape)
    for l in range(1, h.L + 1):
        prod = 1.0
        for d in range(h.D):
            S, t = region.axis_norm_and_tails(h, l, d)
            prod *= S
            assert t[0] <= S and np.all(np.diff(t) <= 1e-15)
            # geometric decay of the inverse mass matrix (ratio 2 - sqrt 3 on
            # a uniform grid): far tails vanish
            assert t[-1] <= S * 1e-12
        assert abs(prod - bounds.K(h, l)) <= 1e-12 * prod
        T = region.tail_bounds(h, l)
        assert T[0] <= prod * h.D


def test_without_regions_the_widths_are_uniform():
    shape = (17, 17)
    w = region.node_widths(shape, 1.0, [])
    assert np.all(w == bounds.bin_widths(shape, 1.0, math.inf)[0])
    # a box as loose as the background still pays one bit for the far field
    assert region.plan(shape, 1.0, [((3, 3), (6, 6), 1.0)])["k"] == [1]


def test_exponents_follow_the_levels():
    shape = (65,)
    regions = [((30,), (30,), 1e-4)]
    pl = region.plan(shape, 1.0, regions)
    k = region.exponents(shape, 1.0, regions)
    h = grid.hierarchy(shape)
    lev = grid.node_level(h)
    # coarse levels dilate farther in index units: every level-0 node that is
    # a corner of the cell around 30 is tight
    assert k[32] == pl["k"][0] and k[28] == pl["k"][0]
    for x in range(65):
        a, b = pl["boxes"][0][lev[x]][0]
        assert (k[x] == pl["k"][0]) == (a <= x <= b)
    assert 2.0 ** -pl["k"][0] <= (1e-4 - pl["far"]) / 1.0


@pytest.mark.parametrize("shape", [(40, 33), (17, 12, 9)])
def test_round_trip_meets_the_region_tolerances(shape):
    rng = np.random.default_rng(3)
    u = rng.standard_normal(shape).cumsum(axis=0).cumsum(axis=1)
    tol = 1e-2 * float(np.max(np.abs(u)))
    lo = tuple(n // 4 for n in shape)
    hi = tuple(n // 2 for n in shape)
    regions = [(lo, hi, tol / 50), (tuple(0 for _ in shape), tuple(2 for _ in shape), tol / 7)]
    q, w = region.compress(u, tol, regions)
    err = np.abs(region.decompress(q, w) - u)
    assert np.all(err <= region.tolerance_map(shape, tol, regions))
    sl = tuple(slice(a, b + 1) for a, b in zip(lo, hi))
    assert np.max(err[sl]) <= tol / 50
