"""Learned tolerance predictor: training data, training and evaluation.

Ratio-targeted compression asks for the relative tolerance tau whose
compressed size is field_bytes / target_ratio.  The network (kernels in
``csrc/mlp.cu``) maps statistics of the field's multilevel coefficients and
log10(target_ratio) to log10(tau); ``mgard_compress_to_ratio`` probes its
proposal and corrects it by bisection when needed, so the error bound is
always the one of the tolerance finally used.

Training data come from the method itself: for every training field one
decomposition (the sizer) gives the exact compressed size at every
tolerance of a log-spaced sweep, and each (field, tolerance) pair is one
sample: input = the field's features with log10 of the ratio reached,
target = log10(tau).  Everything numeric runs in the library's kernels;
this module only orders the calls.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import binding

TAUS = np.logspace(-6.0, 0.0, 32)


def sweep(field: torch.Tensor, taus=TAUS, s: float = math.inf):
    """Samples of one field: (features [len(taus), NFEAT] on the device,
    targets log10(tau) [len(taus)], ratios reached)."""
    sz = binding.Sizer(field, s)
    fbytes = field.numel() * field.element_size()
    xs = torch.empty((len(taus), binding.NFEAT), dtype=torch.float32, device=field.device)
    ratios = []
    for k, tau in enumerate(taus):
        r = fbytes / sz.size(float(tau))
        ratios.append(r)
        sz.features(r, out=xs[k])
    sz.close()
    t = torch.tensor([math.log10(float(tau)) for tau in taus], dtype=torch.float32,
                     device=field.device)
    return xs, t, ratios


def samples(field: torch.Tensor, taus=TAUS, s: float = math.inf):
    """Training samples of one field.  Tolerances below the point where the
    ratio starts to rise are dropped: there many tolerances give the same
    ratio and the inverse map the network learns is undefined."""
    x, t, r = sweep(field, taus, s)
    keep = [k for k in range(len(r)) if r[k] > 1.02 * r[0] and (k == 0 or r[k] > 1.002 * r[k - 1])]
    idx = torch.tensor(keep, dtype=torch.long, device=x.device)
    return x[idx], t[idx]


def dataset(fields, taus=TAUS, s: float = math.inf):
    xs, ts = [], []
    for f in fields:
        x, t = samples(f, taus, s)
        xs.append(x)
        ts.append(t)
    return torch.cat(xs), torch.cat(ts)


def train(x: torch.Tensor, t: torch.Tensor, steps: int = 3000, lr: float = 2e-3, seed: int = 0):
    """Full-batch Adam on the mean squared error of log10(tau).  Returns
    (parameters, losses per step)."""
    p = binding.mlp_init(seed, device=x.device)
    binding.mlp_set_norm(p, x)
    m = torch.zeros(binding.MLP_NTRAIN, dtype=torch.float32, device=x.device)
    v = torch.zeros_like(m)
    losses = binding.mlp_train(p, m, v, x, t, steps, 0, lr)
    return p, losses


def evaluate(fields, targets, params, s: float = math.inf, rel_err: float = 0.05):
    """Ratio targeting with and without the network on every (field, target):
    tolerance probes, time and the ratio error reached (one row per case)."""
    rows = []
    for f in fields:
        fbytes = f.numel() * f.element_size()
        for target in targets:
            row = {"target": target}
            for name, prm in (("predictor", params), ("bisection", None)):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                buf, tol, passes = binding.compress_to_ratio(f, target, s, prm, rel_err)
                torch.cuda.synchronize()
                row[name] = {"passes": passes, "ms": (time.perf_counter() - t0) * 1e3, "tol": tol,
                             "ratio_error": abs(fbytes / buf.numel() / target - 1.0)}
            rows.append(row)
    return rows


def bisect_full(field: torch.Tensor, target: float, s: float = math.inf, rel_err: float = 0.05,
                lo: float = 1e-7, hi: float = 1.0, out=None):
    """Reference search: bisection on log10(tau) where every probe is a
    complete mgard_compress.  Returns (buffer view, tol, passes)."""
    fbytes = field.numel() * field.element_size()
    if out is None:
        out = torch.empty(binding.compress_bound(field.shape, field.dtype), dtype=torch.uint8,
                          device=field.device)
    best = None
    passes = 0

    def probe(tol):
        nonlocal best, passes
        buf = binding.compress(field, tol, s, binding.REL, out=out)
        passes += 1
        r = fbytes / buf.numel()
        e = abs(r / target - 1.0)
        if best is None or e < best[0]:
            best = (e, tol)
        return r

    probe(lo)
    probe(hi)
    for _ in range(60):
        if best[0] <= rel_err or hi / lo <= 1.0 + 1e-9:
            break
        mid = math.sqrt(lo * hi)
        if probe(mid) < target:
            lo = mid
        else:
            hi = mid
    buf = binding.compress(field, best[1], s, binding.REL, out=out)
    return buf, best[1], passes
