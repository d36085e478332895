"""GPU parity of out-of-core compression: every block's buffer equals an
in-core compression of that block alone (whose parity with the oracle the
other tests establish) byte for byte, the reconstruction keeps the bound at
every node against the FP64 input, relative tolerances use max|u| of the
whole field, and corrupt or short buffers are rejected."""
import math

import numpy as np
import pytest
import torch

from oracle import ooc
from paper_2401_05994_b300 import binding, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _field(shape, dtype, seed):
    if len(shape) == 3 and min(shape) > 8:
        u = synth.gaussian_random_field(shape, seed=seed, out_dtype=torch.float64)
    else:
        u = torch.from_numpy(np.random.default_rng(seed).standard_normal(shape).cumsum(axis=0))
    return u.to(dtype).numpy()


@pytest.mark.parametrize("shape,nb,dtype", [
    ((129, 65, 33), 4, np.float32), ((129, 65, 33), 1, np.float32), ((65, 40, 17), 3, np.float64),
    ((5, 33, 17), 5, np.float32), ((300, 200), 7, np.float32), ((4097,), 3, np.float64),
    ((9, 10, 11, 12), 2, np.float32)])
def test_blocks_equal_in_core_compressions(shape, nb, dtype):
    u = _field(shape, torch.float32 if dtype == np.float32 else torch.float64, nb)
    tol = 1e-3 * float(np.max(np.abs(u)))
    buf = binding.compress_ooc(u, tol, nb)
    meta = binding.info(buf)
    assert meta["shape"] == tuple(shape) and meta["tol_abs"] == tol
    ranges = ooc.block_ranges(shape[0], nb)
    spans = binding.ooc_blocks(buf)
    assert len(spans) == nb
    for (a, b), (o0, o1) in zip(ranges, spans):
        ref = binding.compress(torch.from_numpy(np.ascontiguousarray(u[a:b])).to(DEV), tol, math.inf,
                               binding.ABS).cpu().numpy()
        got = buf[o0:o0 + ref.size]
        assert np.array_equal(got, ref), (a, b)
        assert np.all(buf[o0 + ref.size:o1] == 0)
    out = binding.decompress(buf)
    assert out.dtype == u.dtype and out.shape == u.shape
    assert np.max(np.abs(out.astype(np.float64) - u.astype(np.float64))) <= tol


def test_relative_tolerance_uses_the_whole_field():
    u = _field((65, 33, 17), torch.float32, 3)
    u[60, 5, 5] = 40.0   # the maximum sits in the last block
    buf = binding.compress_ooc(u, 1e-3, 4, binding.REL)
    assert binding.info(buf)["tol_abs"] == 1e-3 * 40.0
    out = binding.decompress(buf)
    assert np.max(np.abs(out - u)) <= 1e-3 * 40.0


def test_pinned_buffers_and_rejections():
    shape = (97, 33, 20)
    u = torch.from_numpy(_field(shape, torch.float32, 4)).pin_memory()
    bound = binding.compress_ooc_bound(shape, torch.float32, 3)
    out = torch.empty(bound, dtype=torch.uint8).pin_memory()
    buf = binding.compress_ooc(u, 1e-2, 3, out=out)
    ref = binding.compress_ooc(u.numpy(), 1e-2, 3)
    assert np.array_equal(buf.numpy(), ref)
    with pytest.raises(binding.MgardError) as e:
        binding.compress_ooc(u, 1e-2, 3, out=np.empty(ref.size - 1, np.uint8))
    assert e.value.status == 10
    with pytest.raises(binding.MgardError) as e:
        binding.compress_ooc(u, 1e-2, 98)   # more blocks than planes
    assert e.value.status == 1
    bad = ref.copy()
    bad[88:96] = 255   # first block offset
    with pytest.raises(binding.MgardError) as e:
        binding.decompress(bad)
    assert e.value.status == 7
    with pytest.raises(TypeError):
        binding.compress_ooc(u.cuda(), 1e-2, 3)
