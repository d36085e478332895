"""GPU parity of region-adaptive bounds with the oracle, through the C ABI:
the radius and exponents of the plan, every node's width exponent (bit
exact), and the reconstruction error against each box's tolerance and the
background tolerance; region buffers through the host path, mgard_info and
corrupt headers."""
import math

import numpy as np
import pytest
import torch

from oracle import region
from paper_2401_05994_b300 import binding, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"

CASES = [
    ((65,), 1.0, [((20,), (30,), 1e-2), ((50,), (52,), 1e-3)]),
    ((17, 17), 1.0, [((4, 5), (8, 9), 1e-2), ((12, 0), (16, 3), 1e-3)]),
    ((33, 1, 9), 2.0, [((10, 0, 3), (12, 0, 5), 1e-2)]),
    ((65, 65, 65), 1.0, [((10, 20, 30), (20, 25, 40), 1e-3), ((40, 0, 0), (64, 10, 64), 1e-1)]),
    ((47, 65, 33), 0.5, [((0, 0, 0), (5, 5, 5), 1e-4)]),
    ((9, 10, 11, 12), 1.0, [((2, 3, 4, 5), (4, 5, 6, 7), 1e-2)]),
    ((1025,), 1.0, [((500,), (520,), 1e-3)]),
    ((300, 200), 1.0, [((100, 50), (140, 90), 1e-3), ((0, 150), (40, 199), 3e-2)]),
]


@pytest.mark.parametrize("shape,tol,regions", CASES)
def test_plan_and_exponents_match_oracle(shape, tol, regions):
    rho, k = binding.region_plan(shape, tol, regions)
    pl = region.plan(shape, tol, regions)
    assert rho == pl["rho"] and k == pl["k"]
    got = binding.region_exponents(shape, tol, regions).cpu().numpy()
    assert np.array_equal(got, region.exponents(shape, tol, regions))


def _field(shape, dtype, seed):
    if len(shape) == 3 and min(shape) > 8:
        u = synth.gaussian_random_field(shape, seed=seed, out_dtype=torch.float64)
    else:
        u = torch.from_numpy(np.random.default_rng(seed).standard_normal(shape).cumsum(axis=0))
    return u.to(dtype)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("case", [3, 4, 5, 7])
def test_round_trip_meets_every_tolerance(case, dtype):
    shape, _, regions = CASES[case]
    u = _field(shape, dtype, case).to(DEV)
    umax = float(u.abs().max())
    tol = 1e-2 * umax
    regions = [(lo, hi, t * tol) for lo, hi, t in regions]
    buf = binding.compress_regions(u, tol, regions)
    meta = binding.info(buf)
    assert meta["shape"] == tuple(shape) and meta["tol_abs"] == tol
    out = binding.decompress(buf)
    err = (out.double() - u.double()).abs().cpu().numpy()
    tmap = region.tolerance_map(shape, tol, regions)
    assert np.all(err <= tmap), float(np.max(err / tmap))
    # the tight boxes cost bytes, but only near them
    plain = binding.compress(u, tol, math.inf, binding.ABS)
    assert buf.numel() > plain.numel()


def test_without_boxes_the_inner_buffer_is_the_plain_one():
    u = _field((65, 65, 65), torch.float32, 9).to(DEV)
    buf = binding.compress_regions(u, 0.01, [])
    plain = binding.compress(u, 0.01, math.inf, binding.ABS)
    inner = buf[buf.numel() - plain.numel():]
    assert torch.equal(inner, plain)
    assert torch.equal(binding.decompress(buf), binding.decompress(plain))


def test_host_buffers_and_corrupt_headers():
    shape = (33, 40, 29)
    u = _field(shape, torch.float32, 11)
    regions = [((5, 5, 5), (10, 12, 9), 1e-4)]
    buf = binding.compress_regions(u.to(DEV), 1e-2, regions)
    host = buf.cpu().numpy()
    out = binding.decompress(host)
    err = np.abs(out.astype(np.float64) - u.double().numpy())
    assert np.all(err <= region.tolerance_map(shape, 1e-2, regions))
    assert np.array_equal(out, binding.decompress(buf).cpu().numpy())
    bad = buf.clone()
    bad[12:16] = 255   # nregions
    with pytest.raises(binding.MgardError) as e:
        binding.decompress(bad)
    assert e.value.status == 7
    bad = host.copy()
    bad[16:20] = np.frombuffer(np.int32(99).tobytes(), np.uint8)   # rho beyond the table
    with pytest.raises(binding.MgardError) as e:
        binding.decompress(bad)
    assert e.value.status == 7


def test_bad_regions_are_rejected():
    shape = (33, 33)
    u = torch.ones(shape, device=DEV)
    for regions in ([((0, 0), (33, 3), 1e-3)],            # outside the field
                    [((5, 5), (3, 8), 1e-3)],             # empty
                    [((0, 0), (3, 3), 2.0)],              # looser than the background
                    [((0, 0), (3, 3), 1e-30)],            # beyond 2^-60
                    [((0, 0), (1, 1), 1e-3)] * 9):        # too many
        with pytest.raises(binding.MgardError) as e:
            binding.compress_regions(u, 1.0, regions)
        assert e.value.status == 1, regions
