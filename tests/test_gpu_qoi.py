"""GPU parity of linear-QoI error control with the oracle, through the C ABI:
the representer, the dual norm for finite and infinite s, the QoI value, and
QoI-controlled compression (its tolerance, its bytes against a plain
compression at that tolerance, and the QoI's error after decompression)."""
import math

import numpy as np
import pytest
import torch

from oracle import qoi
from paper_2401_05994_b300 import binding, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"

SHAPES = [(65,), (33, 20), (17, 9, 12), (9, 6, 5, 7), (5, 1, 9), (2, 3)]


def _weights(shape, kind, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "random":
        return rng.standard_normal(shape)
    if kind == "positive":
        return rng.uniform(0.0, 1.0, shape) / np.prod(shape)
    g = np.zeros(shape)
    box = tuple(slice(n // 4, max(n // 4 + 1, 3 * n // 4)) for n in shape)
    g[box] = 1.0
    return g / g.sum()


@pytest.mark.parametrize("shape", SHAPES)
def test_representer_matches_oracle(shape):
    g = _weights(shape, "random", 1)
    r = binding.qoi_representer(torch.from_numpy(g).to(DEV)).cpu().numpy()
    ref = qoi.representer(g)
    assert np.max(np.abs(r - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("s", [0.0, 0.5, 1.0, math.inf])
def test_dual_norm_matches_oracle(shape, s):
    for kind in ("random", "box"):
        g = _weights(shape, kind, 2)
        got = binding.qoi_norm(torch.from_numpy(g).to(DEV), s)
        ref = qoi.norm(g, s)
        assert abs(got - ref) <= 1e-10 * ref, (kind, got, ref)


def test_integral_functional_on_the_device():
    shape = (33, 17, 9)
    w = np.ones(())
    for n in shape:
        a = np.ones(n)
        a[0] = a[-1] = 0.5
        w = np.multiply.outer(w, a)
    g = torch.from_numpy(w).to(DEV)
    r = binding.qoi_representer(g)
    assert float((r - 1.0).abs().max()) < 1e-12
    vol = 32.0 * 16.0 * 8.0
    for s in (0.0, 1.0):
        assert abs(binding.qoi_norm(g, s) - math.sqrt(vol)) < 1e-10 * math.sqrt(vol)
    assert binding.qoi_norm(g, math.inf) == vol


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_value_matches_oracle(dtype):
    shape = (47, 33, 20)
    u = synth.gaussian_random_field(shape, seed=3, out_dtype=torch.float64).to(dtype)
    g = _weights(shape, "random", 4)
    got = binding.qoi_value(u.to(DEV), torch.from_numpy(g).to(DEV))
    ref = qoi.value(u.double().numpy(), g)
    assert abs(got - ref) <= 1e-12 * np.sum(np.abs(g)) * float(u.abs().max())


@pytest.mark.parametrize("s", [0.0, 1.0, math.inf])
def test_compress_qoi_meets_the_qoi_tolerance(s):
    shape = (65, 65, 65)
    u = synth.gaussian_random_field(shape, seed=5).to(DEV)
    umax = float(u.abs().max())
    for kind in ("box", "positive", "random"):
        g64 = _weights(shape, kind, 6)
        g = torch.from_numpy(g64).to(DEV)
        q0 = binding.qoi_value(u, g)
        for rel in (1e-2, 1e-4):
            tol = rel * umax * float(np.sum(np.abs(g64)))
            buf, tol_used = binding.compress_qoi(u, g, tol, s)
            assert abs(tol_used - tol / qoi.norm(g64, s)) <= 1e-10 * tol_used
            plain = binding.compress(u, tol_used, s, binding.ABS)
            assert torch.equal(buf, plain)
            err = abs(binding.qoi_value(binding.decompress(buf), g) - q0)
            assert err <= tol, (kind, rel, err / tol)


def test_bad_weights_are_rejected():
    shape = (17, 9)
    g = torch.zeros(shape, dtype=torch.float64, device=DEV)
    u = torch.ones(shape, device=DEV)
    with pytest.raises(binding.MgardError) as e:
        binding.compress_qoi(u, g, 1e-3, 0.0)
    assert e.value.status == 1
    g[3, 4] = float("nan")
    with pytest.raises(binding.MgardError) as e:
        binding.qoi_norm(g, 0.0)
    assert e.value.status == 4
    g[3, 4] = 1.0
    with pytest.raises(binding.MgardError) as e:
        binding.qoi_norm(g, -1.0)
    assert e.value.status == 1
    with pytest.raises(TypeError):
        binding.qoi_norm(g.cpu(), 0.0)
