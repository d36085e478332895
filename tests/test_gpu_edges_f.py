"""Degenerate cases of the QoI, region-adaptive and out-of-core paths: a
grid of one node, blocks of one plane or one node, a box over the whole
field, the smallest grids with a level."""
import math

import numpy as np
import pytest
import torch

from oracle import qoi, region
from paper_2401_05994_b300 import binding

pytestmark = pytest.mark.gpu
DEV = "cuda"


def test_qoi_on_a_single_node():
    g = torch.full((1, 1, 1), 2.5, dtype=torch.float64, device=DEV)
    for s in (0.0, 1.0, math.inf):
        assert binding.qoi_norm(g, s) == qoi.norm(g.cpu().numpy(), s) == 2.5
    u = torch.full((1, 1, 1), 3.0, device=DEV)
    buf, tol = binding.compress_qoi(u, g, 1e-3, 0.0)
    assert tol == 1e-3 / 2.5
    err = abs(binding.qoi_value(binding.decompress(buf), g) - binding.qoi_value(u, g))
    assert err <= 1e-3


@pytest.mark.parametrize("shape,nb", [((3,), 3), ((5, 4), 5), ((2, 33), 2), ((7, 1, 9), 7)])
def test_out_of_core_blocks_of_one_plane(shape, nb):
    u = np.random.default_rng(nb).standard_normal(shape).astype(np.float32)
    tol = 1e-2
    buf = binding.compress_ooc(u, tol, nb)
    out = binding.decompress(buf)
    assert out.shape == u.shape
    assert np.max(np.abs(out.astype(np.float64) - u)) <= tol


def test_region_over_the_whole_field():
    shape = (33, 17)
    u = torch.from_numpy(np.random.default_rng(2).standard_normal(shape).cumsum(axis=0)).float().to(DEV)
    regions = [((0, 0), (32, 16), 1e-3)]
    buf = binding.compress_regions(u, 1e-1, regions)
    err = (binding.decompress(buf).double() - u.double()).abs().max().item()
    assert err <= 1e-3
    k = binding.region_exponents(shape, 1e-1, regions).cpu().numpy()
    assert np.all(k == region.exponents(shape, 1e-1, regions))
    assert np.all(k == region.plan(shape, 1e-1, regions)["k"][0])


@pytest.mark.parametrize("shape", [(3,), (3, 3), (3, 3, 3)])
def test_regions_on_the_smallest_grids_with_a_level(shape):
    u = torch.from_numpy(np.random.default_rng(3).standard_normal(shape)).float().to(DEV)
    lo = tuple(0 for _ in shape)
    regions = [(lo, lo, 1e-4)]
    buf = binding.compress_regions(u, 1e-2, regions)
    err = (binding.decompress(buf).double() - u.double()).abs().cpu().numpy()
    assert np.all(err <= region.tolerance_map(shape, 1e-2, regions))
    assert err[lo] <= 1e-4


def test_regions_need_a_level():
    u = torch.zeros((2, 3, 3), device=DEV)   # an axis of two nodes: no levels
    with pytest.raises(binding.MgardError) as e:
        binding.compress_regions(u, 1e-2, [((0, 0, 0), (0, 0, 0), 1e-4)])
    assert e.value.status == 2
