"""Batched compression (mgard_compress_batch) against single-field compression.

Every field of a batch must come out byte for byte as mgard_compress makes
it (the per-field pipeline is the same; the batch only changes the streams
and, with graph capture, how the launches are issued), and decompress within
its bound against the FP64 oracle's error measure.
"""
import math

import numpy as np
import pytest
import torch

from oracle import pipeline
from paper_2401_05994_b300 import binding, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"

SHAPES = [(33, 40, 29), (65, 17, 9), (100,), (9, 257), (5, 6, 7, 8), (47, 33, 65), (3, 3, 3)]


def _fields(dtype=torch.float32, shapes=SHAPES, seed=100):
    out = []
    for k, sh in enumerate(shapes):
        if len(sh) == 3 and min(sh) > 4:
            u = synth.gaussian_random_field(sh, seed=seed + k, beta=2.0 + (k % 3) * 0.8)
        else:
            u = torch.from_numpy(np.random.default_rng(seed + k).standard_normal(sh))
        out.append(u.to(dtype).to(DEV).contiguous())
    return out


def _single(f, tol, s, mode):
    buf = binding.compress(f, tol, s, mode)
    return buf.cpu().numpy()


@pytest.mark.parametrize("s", [math.inf, 0.0, 1.0])
@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("persistent", [False, True])
def test_batch_bytes_equal_single(s, graph, persistent):
    fields = _fields()
    ref = [_single(f, 1e-3, s, binding.REL) for f in fields]
    outs = [torch.empty(binding.compress_bound(f.shape), dtype=torch.uint8, device=DEV) for f in fields]
    for _ in range(2):   # the second graph call replays the captured graph
        for o in outs:
            o.fill_(0xAB)
        views, sizes, stats = binding.compress_batch(fields, 1e-3, s, binding.REL, outs=outs,
                                                     graph=graph, persistent=persistent)
        assert stats == [0] * len(fields)
        for v, z, r in zip(views, sizes, ref):
            assert z == len(r)
            assert np.array_equal(v.cpu().numpy(), r)


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_graph_replay_sees_new_data(persistent):
    fields = _fields(shapes=[(33, 33, 33), (17, 65, 9)])
    outs = [torch.empty(binding.compress_bound(f.shape), dtype=torch.uint8, device=DEV) for f in fields]
    binding.compress_batch(fields, 1e-3, math.inf, binding.REL, outs=outs, graph=True,
                           persistent=persistent)
    # same buffers, new contents: the replayed graph must read them
    for k, f in enumerate(fields):
        f.copy_(synth.gaussian_random_field(tuple(f.shape), seed=900 + k).to(DEV))
    views, sizes, _ = binding.compress_batch(fields, 1e-3, math.inf, binding.REL, outs=outs, graph=True,
                                             persistent=persistent)
    for f, v in zip(fields, views):
        assert np.array_equal(v.cpu().numpy(), _single(f, 1e-3, math.inf, binding.REL))


@pytest.mark.parametrize("s", [math.inf, 0.0])
def test_batch_error_bound(s):
    fields = _fields(dtype=torch.float64, shapes=[(33, 40, 29), (65, 17, 9), (129,)])
    views, _, _ = binding.compress_batch(fields, 1e-4, s, binding.ABS, graph=True)
    for f, v in zip(fields, views):
        out = binding.decompress(v)
        err = pipeline.error(f.cpu().numpy(), out.cpu().numpy(), s)
        assert err <= binding.info(v)["tol_abs"]


@pytest.mark.parametrize("persistent", [False, True])
def test_batch_capacity_and_nonfinite_per_field(persistent):
    fields = _fields(shapes=[(33, 33, 33), (20, 20, 20), (40, 9, 9)])
    fields[2][1, 2, 3] = float("nan")
    outs = [torch.empty(binding.compress_bound(f.shape), dtype=torch.uint8, device=DEV) for f in fields]
    need = len(_single(fields[1], 1e-3, math.inf, binding.REL))
    outs[1] = torch.empty(need - 64, dtype=torch.uint8, device=DEV)
    _, sizes, stats = binding.compress_batch(fields, 1e-3, math.inf, binding.REL, outs=outs,
                                             check=False, persistent=persistent)
    assert stats[0] == 0
    assert stats[1] == 10   # MGARD_ECAPACITY
    assert sizes[1] == need
    assert stats[2] == 4    # MGARD_ENONFINITE
    with pytest.raises(binding.MgardError):
        binding.compress_batch(fields, 1e-3, math.inf, binding.REL, outs=outs)


def test_batch_rejects_host_buffers():
    f = torch.zeros(33, 33)
    with pytest.raises(Exception):
        binding.compress_batch([f], 1e-3)


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("persistent", [False, True])
def test_decompress_batch_equals_single(graph, persistent):
    fields = _fields()
    views, _, _ = binding.compress_batch(fields, 1e-3, math.inf, binding.REL)
    bufs = [v.clone() for v in views]
    ref = [binding.decompress(b).cpu().numpy() for b in bufs]
    outs = [torch.full(f.shape, 7.0, dtype=f.dtype, device=DEV) for f in fields]
    for _ in range(2):   # graph replay on the second call
        got, stats = binding.decompress_batch(bufs, outs=outs, graph=graph, persistent=persistent)
        assert stats == [0] * len(bufs)
        for g, r in zip(got, ref):
            assert np.array_equal(g.cpu().numpy(), r)


def test_decompress_batch_per_buffer_failures():
    fields = _fields(shapes=[(33, 33, 33), (20, 20, 20), (40, 9, 9)])
    views, _, _ = binding.compress_batch(fields, 1e-3, math.inf, binding.REL)
    bufs = [v.clone() for v in views]
    bufs[0][0] ^= 0xFF                     # magic
    outs = [torch.empty(f.shape, dtype=f.dtype, device=DEV) for f in fields]
    outs[1] = torch.empty(100, dtype=torch.float32, device=DEV)   # too small
    got, stats = binding.decompress_batch(bufs, outs=outs, check=False)
    assert stats[0] == 7    # MGARD_ECORRUPT
    assert stats[1] == 10   # MGARD_ECAPACITY
    assert stats[2] == 0
    assert np.array_equal(got[2].cpu().numpy(), binding.decompress(bufs[2]).cpu().numpy())
    # a corrupt payload is found by the decoder, not only by header checks
    bad = bufs[2].clone()
    bad[-64:] = 0x5A
    _, stats = binding.decompress_batch([bad], outs=[outs[2]], check=False)
    assert stats[0] in (0, 7)   # flipped payload bits may still decode to valid codes


def test_autotune_keeps_bits():
    f = _fields(shapes=[(65, 47, 33)])[0]
    before = _single(f, 1e-3, math.inf, binding.REL)
    rep = binding.autotune(f.shape)
    assert "level" in rep
    after = _single(f, 1e-3, math.inf, binding.REL)
    assert np.array_equal(before, after)
    out = binding.decompress(torch.from_numpy(after).to(DEV))
    assert pipeline.error(f.cpu().numpy().astype(np.float64), out.cpu().numpy().astype(np.float64),
                          math.inf) <= binding.info(after)["tol_abs"]
