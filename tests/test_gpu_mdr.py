"""GPU parity of refactoring (MDRefactor / MDRequest / MDReconstruct) with
the oracle, through the C ABI.

* The bit planes are bit-exact with the oracle's encoding of the library's
  own coefficients (the library decomposes in float32; its in-place
  decomposition gives the same coefficients as the level-order one the
  refactoring uses).
* Requests equal the oracle's greedy choice on the same header.
* Reconstructions equal the oracle's FP64 decoding and recomposition of the
  same planes to float32 rounding, and their error against the input stays
  within the estimate plus float32 rounding.
"""
import math

import numpy as np
import pytest
import torch

from oracle import bounds, grid, mdr, multilevel
from paper_2401_05994_b300 import binding, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"

SHAPES = [(65, 65, 65), (47, 65, 33), (33, 20), (1000,), (129, 9, 40)]


def _field(shape, dtype, seed):
    if len(shape) >= 2 and min(shape) > 8:
        u = synth.gaussian_random_field(shape, seed=seed, out_dtype=torch.float64)
    else:
        u = torch.from_numpy(np.random.default_rng(seed).standard_normal(shape).cumsum(axis=-1))
    return u.to(dtype)


def _levels_from_buffer(buf, h):
    host = buf.cpu().numpy()
    B = h["planes"]
    out = []
    for lv in h["levels"]:
        nw = lv["words"]
        w = host[lv["offset"]:lv["offset"] + 4 * (B + 1) * nw].view(np.uint32)
        out.append((w[:nw], [w[(1 + b) * nw:(2 + b) * nw] for b in range(B)]))
    return out


def _oracle_record(h, planes_lv, shape):
    return dict(shape=shape, B=h["planes"], max_levels=None,
                counts=[lv["count"] for lv in h["levels"]],
                exponents=[lv["exponent"] for lv in h["levels"]],
                signs=[p[0] for p in planes_lv], planes=[p[1] for p in planes_lv],
                nonzero=[lv["nonzero"] for lv in h["levels"]],
                weights=[lv["weight"] for lv in h["levels"]])


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape", SHAPES)
def test_planes_bit_exact_with_oracle_encoding(shape, dtype):
    u = _field(shape, dtype, 31).to(DEV)
    B = 32 if dtype == torch.float32 else 24
    buf, h = binding.refactor(u, B)
    assert h["magic"] == b"MGARDMDR" and h["planes"] == B and h["total_bytes"] == buf.numel()
    assert h["shape"] == tuple(shape)
    assert h["max_abs"] == float(u.abs().max())
    coeff = multilevel.level_coefficients(binding.decompose(u.clone()).cpu().double().numpy())
    hh = grid.hierarchy(shape)
    assert len(coeff) == h["nlevels"] == hh.L + 1
    planes_lv = _levels_from_buffer(buf, h)
    for l, (c, lv, (signs, planes)) in enumerate(zip(coeff, h["levels"], planes_lv)):
        e, rs, rp = mdr.encode_level(c, B)
        assert lv["count"] == len(c) and lv["exponent"] == e and lv["nonzero"] == bool(np.any(c))
        assert np.array_equal(signs, rs)
        for b in range(B):
            assert np.array_equal(planes[b], rp[b]), (l, b)
        w = 1.0 if l == 0 else bounds.linf_level_constant(hh, l)
        assert abs(lv["weight"] - w) <= 1e-12 * w


@pytest.mark.parametrize("shape", [(65, 65, 65), (33, 20)])
def test_request_and_reconstruct_match_oracle(shape):
    u = _field(shape, torch.float32, 32).to(DEV)
    buf, h = binding.refactor(u, 32)
    r = _oracle_record(h, _levels_from_buffer(buf, h), shape)
    un = u.cpu().double().numpy()
    umax = float(np.max(np.abs(un)))
    for rel in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5):
        tol = rel * umax
        P, nbytes, est = binding.request(h, tol)
        rP, rbytes, rest = mdr.request(r, tol)
        assert P == rP and nbytes == rbytes and est == rest and est <= tol
        got = binding.reconstruct(buf, P).cpu().double().numpy()
        ref = mdr.reconstruct(r, P)
        assert np.max(np.abs(got - ref)) <= 2e-5 * max(1.0, umax)
        # against the input: the estimate plus the float32 rounding of the
        # decomposition and recomposition
        assert np.max(np.abs(got - un)) <= est + 1e-5 * umax
        assert np.max(np.abs(ref - un)) <= est + 1e-5 * umax
    # fewer bytes for looser tolerances, and every plane recovers the field
    sizes = [binding.request(h, t * umax)[1] for t in (1e-1, 1e-3, 1e-5)]
    assert sizes == sorted(sizes) and sizes[0] < sizes[-1]
    full = binding.reconstruct(buf, [32] * h["nlevels"]).cpu().double().numpy()
    assert np.max(np.abs(full - un)) <= 1e-5 * umax


def test_request_below_every_plane_and_bad_inputs():
    u = _field((33, 33, 33), torch.float32, 33).to(DEV)
    buf, h = binding.refactor(u, 8)
    P, nbytes, est = binding.request(h, 0.0)   # MGARD_EBOUND: every plane
    assert all(p == (8 if lv["nonzero"] else 0) for p, lv in zip(P, h["levels"]))
    assert nbytes == sum(4 * lv["words"] * 9 for lv in h["levels"] if lv["nonzero"])
    assert est > 0.0
    with pytest.raises(binding.MgardError) as e:
        binding.refactor(torch.zeros((9, 6, 5, 7), device=DEV), 8)
    assert e.value.status == 2
    bad = buf.clone()
    bad[0] ^= 0xFF
    with pytest.raises(binding.MgardError) as e:
        binding.reconstruct(bad, P)
    assert e.value.status == 7
    with pytest.raises(binding.MgardError) as e:
        binding.reconstruct(buf, [9] * h["nlevels"])
    assert e.value.status == 1
    nan = u.clone()
    nan[1, 2, 3] = float("nan")
    with pytest.raises(binding.MgardError) as e:
        binding.refactor(nan, 8)
    assert e.value.status == 4
