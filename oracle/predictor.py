"""Tolerance predictor: features, MLP and Adam (oracle; test infrastructure).

A small multilayer perceptron maps statistics of a field's multilevel
coefficients plus a target compression ratio to log10 of the relative
tolerance that reaches the ratio.  The paper has no predictor; everything
here is a reading written from the standard definitions:

Features (``features``), per level l = L, L-1, ... (finest first, at most
``NLEV`` levels; missing slots are zero), over that level's coefficients c
(level 0: its nodal values), with a = max|u| of the field:

* log10 of the number of coefficients,
* mean and standard deviation (population) of r = log10(max(|c|, 1e-12 a) / a),
* for j = 0..14 the fraction of coefficients with |c| < 10^(-j/2) a;

then four global inputs: number of active axes D, L, log10 N and
log10(target ratio).  ``NFEAT = NLEV * 18 + 4 = 220``.

Network (``forward``): x is standardized with per-input mean mu and standard
deviation sd, floored at SD_FLOOR = 0.05 so that inputs that barely vary in
the training set do not turn small differences into large inputs, then
h1 = relu(W1 xn + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3, with
64 hidden units per layer and relu'(0) = 0.  Loss: mean squared error
(1/B) sum_b (y_b - t_b)^2.  ``loss_grad`` is hand-written backpropagation;
``adam_step`` is Adam (Kingma & Ba 2015) with bias correction.

Parameter vector layout (float): W1 [H, IN] row-major, b1 [H], W2 [H, H],
b2 [H], w3 [H], b3 [1] (the trainable part, ``ntrain``), then mu [IN] and
sd [IN].
"""
from __future__ import annotations

import numpy as np

from .multilevel import level_coefficients

NLEV = 12
NTHR = 15
PER_LEVEL = 3 + NTHR
NGLOBAL = 4
NFEAT = NLEV * PER_LEVEL + NGLOBAL
H = 64


def features(v: np.ndarray, umax: float, D: int, target_ratio: float, max_levels=None):
    """Feature vector of an in-place decomposed array ``v`` (see module doc)."""
    levels = level_coefficients(v, max_levels)
    L = len(levels) - 1
    a = float(umax) if umax > 0 else 1.0
    f = np.zeros(NFEAT)
    for slot in range(min(NLEV, L + 1)):
        c = np.abs(np.asarray(levels[L - slot], dtype=np.float64))
        n = c.size
        base = slot * PER_LEVEL
        f[base] = np.log10(n)
        r = np.log10(np.maximum(c, 1e-12 * a) / a)
        f[base + 1] = r.mean()
        f[base + 2] = r.std()
        for j in range(NTHR):
            f[base + 3 + j] = np.count_nonzero(c < 10.0 ** (-j / 2.0) * a) / n
    g = NLEV * PER_LEVEL
    f[g] = D
    f[g + 1] = L
    f[g + 2] = np.log10(np.prod(v.shape))
    f[g + 3] = np.log10(target_ratio)
    return f


def sizes(nin=NFEAT, h=H):
    ntrain = h * nin + h + h * h + h + h + 1
    return ntrain, ntrain + 2 * nin


def unpack(p, nin=NFEAT, h=H):
    p = np.asarray(p, dtype=np.float64)
    o = 0

    def take(k, shape=None):
        nonlocal o
        a = p[o:o + k]
        o += k
        return a.reshape(shape) if shape else a

    W1 = take(h * nin, (h, nin))
    b1 = take(h)
    W2 = take(h * h, (h, h))
    b2 = take(h)
    w3 = take(h)
    b3 = take(1)
    mu = take(nin)
    sd = take(nin)
    return W1, b1, W2, b2, w3, b3, mu, sd


SD_FLOOR = 0.05


def standardize(x, mu, sd):
    return (x - mu) / np.maximum(sd, SD_FLOOR)


def forward(p, x, nin=NFEAT, h=H):
    """Outputs y [B] for inputs x [B, nin]."""
    W1, b1, W2, b2, w3, b3, mu, sd = unpack(p, nin, h)
    xn = standardize(np.asarray(x, dtype=np.float64), mu, sd)
    h1 = np.maximum(xn @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3[0]


def loss_grad(p, x, t, nin=NFEAT, h=H):
    """(loss, gradient over the trainable parameters) of the mean squared
    error, by backpropagation through the three layers."""
    W1, b1, W2, b2, w3, b3, mu, sd = unpack(p, nin, h)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = x.shape[0]
    xn = standardize(x, mu, sd)
    z1 = xn @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3[0]
    e = y - t
    loss = np.mean(e * e)
    dy = 2.0 * e / B                      # dL/dy_b
    gw3 = h2.T @ dy
    gb3 = np.array([dy.sum()])
    d2 = np.outer(dy, w3) * (z2 > 0)      # dL/dz2
    gW2 = d2.T @ h1
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)             # dL/dz1
    gW1 = d1.T @ xn
    gb1 = d1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, gb3])
    return loss, g


def set_norm(p, x, nin=NFEAT, h=H):
    """Parameters with mu, sd set to the per-input mean and population
    standard deviation of x."""
    p = np.array(p, dtype=np.float64)
    ntrain, _ = sizes(nin, h)
    x = np.asarray(x, dtype=np.float64)
    p[ntrain:ntrain + nin] = x.mean(axis=0)
    p[ntrain + nin:] = x.std(axis=0)
    return p


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of the first len(g) entries of p (t counts from 1)."""
    p = np.array(p, dtype=np.float64)
    k = len(g)
    m = b1 * np.asarray(m, dtype=np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    p[:k] -= lr * mh / (np.sqrt(vh) + eps)
    return p, m, v
