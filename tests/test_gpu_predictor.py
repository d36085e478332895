"""Tolerance predictor on the GPU against the FP64 oracle, and what the
trained network gains over plain bisection.

* features of a decomposed field (sizer) against oracle.predictor.features
  on the oracle's decomposition;
* network forward pass, gradient (backpropagation kernels) and Adam step
  against the oracle's FP64 definitions (1e-4 relative);
* the sizer's sizes and buffers against mgard_compress, byte for byte;
* ratio targeting: within 5% with and without the network, and fewer
  tolerance probes with a network trained on earlier timesteps of an
  advected field than bisection needs on later ones.
"""
import math

import numpy as np
import pytest
import torch

from oracle import multilevel, predictor as P
from paper_2401_05994_b300 import binding, predictor, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _field(shape, seed=3, dtype=torch.float64):
    return synth.gaussian_random_field(shape, seed=seed).to(dtype).to(DEV).contiguous()


@pytest.mark.parametrize("shape", [(33, 40, 29), (65, 17), (129,), (5, 6, 7, 9)])
def test_features_match_oracle(shape):
    if len(shape) == 3:
        u = _field(shape)
    else:
        u = torch.from_numpy(np.random.default_rng(5).standard_normal(shape)).to(DEV)
    sz = binding.Sizer(u, math.inf)
    got = sz.features(37.5).cpu().numpy().astype(np.float64)
    sz.close()
    un = u.cpu().numpy()
    ref = P.features(multilevel.decompose(un), float(np.abs(un).max()),
                     sum(1 for n in shape if n > 1), 37.5)
    per = P.PER_LEVEL
    for slot in range(P.NLEV):
        b = slot * per
        assert got[b] == pytest.approx(ref[b], rel=1e-6, abs=1e-6)              # log10 count
        assert got[b + 1] == pytest.approx(ref[b + 1], rel=1e-5, abs=1e-5)      # mean
        assert got[b + 2] == pytest.approx(ref[b + 2], rel=1e-4, abs=1e-4)      # std
        n = 10 ** ref[b] if ref[b] else 1
        # a coefficient within float rounding of a threshold may count on either side
        assert np.max(np.abs(got[b + 3:b + per] - ref[b + 3:b + per])) <= 2.0 / n + 1e-6
    assert np.allclose(got[P.NLEV * per:], ref[P.NLEV * per:], rtol=1e-6)


def _host_params(p):
    return p.cpu().numpy().astype(np.float64)


def test_forward_gradient_adam_match_oracle():
    rng = np.random.default_rng(11)
    B = 48
    x = torch.from_numpy(rng.standard_normal((B, P.NFEAT)).astype(np.float32)).to(DEV)
    x[:, 7] = 3.0                                      # a constant input (sd = 0)
    t = torch.from_numpy(rng.standard_normal(B).astype(np.float32)).to(DEV)
    p = binding.mlp_init(5)
    binding.mlp_set_norm(p, x)
    ph = _host_params(p)
    xh, th = x.cpu().numpy().astype(np.float64), t.cpu().numpy().astype(np.float64)
    # standardization statistics
    assert np.allclose(ph[P.sizes()[0]:P.sizes()[0] + P.NFEAT], xh.mean(0), rtol=1e-5, atol=1e-6)
    y = binding.mlp_forward(p, x).cpu().numpy()
    yr = P.forward(ph, xh)
    assert np.max(np.abs(y - yr)) <= 1e-4 * max(1.0, np.max(np.abs(yr)))
    loss, g = binding.mlp_loss_grad(p, x, t)
    lr_, gr = P.loss_grad(ph, xh, th)
    assert float(loss.item()) == pytest.approx(lr_, rel=1e-4)
    g = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - gr)) <= 1e-4 * np.max(np.abs(gr))
    # one Adam step from zero moments
    m = torch.zeros(binding.MLP_NTRAIN, device=DEV)
    v = torch.zeros_like(m)
    gd = torch.from_numpy(gr.astype(np.float32)).to(DEV)
    binding.adam_step(p, gd, m, v, 1, 1e-3)
    pr, mr, vr = P.adam_step(ph, gr.astype(np.float32).astype(np.float64), np.zeros_like(gr),
                             np.zeros_like(gr), 1, 1e-3)
    assert np.max(np.abs(_host_params(p) - pr)) <= 1e-6


def test_training_reduces_loss_like_oracle():
    # a learnable map of the inputs: the kernels' training matches the
    # oracle's loss curve over a few steps and keeps decreasing
    rng = np.random.default_rng(2)
    B = 64
    xh = rng.standard_normal((B, P.NFEAT))
    th = 0.5 * xh[:, 0] - 0.25 * xh[:, 3] + 0.1
    x = torch.from_numpy(xh.astype(np.float32)).to(DEV)
    t = torch.from_numpy(th.astype(np.float32)).to(DEV)
    p = binding.mlp_init(1)
    binding.mlp_set_norm(p, x)
    ph = _host_params(p)
    m = torch.zeros(binding.MLP_NTRAIN, device=DEV)
    v = torch.zeros_like(m)
    losses = binding.mlp_train(p, m, v, x, t, 5, 0, 1e-3).cpu().numpy()
    ntrain = P.sizes()[0]
    mh, vh = np.zeros(ntrain), np.zeros(ntrain)
    ref = []
    for k in range(1, 6):
        l, g = P.loss_grad(ph, xh.astype(np.float32), th.astype(np.float32))
        ref.append(l)
        ph, mh, vh = P.adam_step(ph, g, mh, vh, k, 1e-3)
    assert np.allclose(losses, ref, rtol=1e-3)
    more = binding.mlp_train(p, m, v, x, t, 400, 5, 1e-3).cpu().numpy()
    assert more[-1] < 0.05 * losses[0]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_sizer_sizes_and_buffers_equal_compress(dtype):
    u = _field((47, 33, 65), dtype=dtype)
    sz = binding.Sizer(u, math.inf)
    for tol in (1e-5, 1e-3, 3e-2):
        ref = binding.compress(u, tol, math.inf, binding.REL)
        assert sz.size(tol) == ref.numel()
        got = sz.compress(tol)
        assert np.array_equal(got.cpu().numpy(), ref.cpu().numpy())
    sz.close()
    v = _field((40, 40, 40), dtype=dtype)
    sz = binding.Sizer(v, 0.0)
    ref = binding.compress(v, 1e-3, 0.0, binding.REL)
    assert sz.size(1e-3) == ref.numel()
    sz.close()


def test_bisection_reaches_target():
    u = _field((64, 96, 96), dtype=torch.float32)
    fbytes = u.numel() * 4
    for target in (3.0, 8.0):
        buf, tol, passes = binding.compress_to_ratio(u, target, math.inf, None, 0.05)
        assert abs(fbytes / buf.numel() / target - 1.0) <= 0.05
        out = binding.decompress(buf)
        err = float((out.double() - u.double()).abs().max())
        assert err <= tol * float(u.abs().max())


def test_predictor_needs_fewer_probes_than_bisection():
    shape = (48, 64, 64)
    fields = [synth.advected_field(shape, t, seed=7, device=DEV).contiguous() for t in range(16)]
    x, t = predictor.dataset(fields[:12])
    params, losses = predictor.train(x, t, steps=3000, lr=2e-3)
    assert float(losses[-1]) < 0.1 * float(losses[0])
    rows = predictor.evaluate(fields[12:], [2.5, 5.0, 8.0], params)
    pp = [r["predictor"]["passes"] for r in rows]
    bp = [r["bisection"]["passes"] for r in rows]
    assert all(r["predictor"]["ratio_error"] <= 0.05 for r in rows)
    assert all(r["bisection"]["ratio_error"] <= 0.05 for r in rows)
    assert np.mean(pp) < 0.5 * np.mean(bp), (pp, bp)
