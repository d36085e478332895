"""Level-wise linear quantization (oracle; test infrastructure).

The paper ("Software design") approximates each multilevel coefficient by an
integer multiple of its level's bin width.  Readings fixed here:

* ``q = rint(c / w)``, ties to even.
* Dictionary of ``DICT = 4096`` symbols, ``R = 2048``: ``|q| < R`` is coded as
  symbol ``q + R`` (1..4095); otherwise symbol 0 (escape) and ``q`` goes to the
  outlier list, in symbol order, as a 32-bit integer.
* Symbol order: level 0 (all of its nodes), then levels 1..L (only the nodes
  new on that level), each in row-major order of that level's grid.
* ``precision="f64"`` decides ``q = rint(c / w)`` in double precision.
  ``precision="f32"`` takes the decision the way a single-precision
  quantizer does: ``x = float32(c) * float32(1/w)`` rounded to float32,
  ``q = rint(x)``; only when ``|q| >= F32_EXACT = 4096`` is the stored value
  recomputed as ``rint(c / w)`` in double precision.
* Dequantization: ``q * w`` in the working precision; for f32 data
  ``float32(q) * float32(w)`` when ``|q| < 4096`` and ``float32(q * w)``
  (double product) otherwise.
"""
from __future__ import annotations

import numpy as np

from .multilevel import level_coefficients
from .grid import hierarchy

DICT = 4096
R = DICT // 2
ESC = 0
QMAX = 2 ** 31 - 1
F32_EXACT = 4096


class ToleranceTooSmall(ValueError):
    pass


def quantize_levels(levels, widths, precision="f64"):
    """Quantize per-level coefficient vectors.

    Returns ``(symbols uint16, outliers int32, hist uint64)``."""
    syms, outs = [], []
    for c, w in zip(levels, widths):
        c = np.asarray(c)
        c64 = c.astype(np.float64)
        if precision == "f32":
            c32 = c.astype(np.float32)
            x = c32 * np.float32(1.0 / w)
            q = np.rint(x).astype(np.float64)
            big = np.abs(q) >= F32_EXACT
            q = np.where(big, np.rint(c64 / w), q)
        else:
            q = np.rint(c64 / w)
        esc = np.abs(q) >= R
        if precision == "f32":
            # the escape decision is the float32 one
            esc = np.abs(np.rint(c.astype(np.float32) * np.float32(1.0 / w))) >= R
        sym = np.where(esc, ESC, q + R).astype(np.uint16)
        qo = q[esc]
        if qo.size and np.max(np.abs(qo)) > QMAX:
            raise ToleranceTooSmall("quantized value exceeds 32-bit range")
        syms.append(sym)
        outs.append(qo.astype(np.int32))
    symbols = np.concatenate(syms) if syms else np.zeros(0, np.uint16)
    outliers = np.concatenate(outs) if outs else np.zeros(0, np.int32)
    hist = np.bincount(symbols, minlength=DICT).astype(np.uint64)
    return symbols, outliers, hist


def quantize(v: np.ndarray, widths, max_levels=None, precision="f64"):
    """Quantize an in-place decomposed array (see module docstring)."""
    return quantize_levels(level_coefficients(v, max_levels), widths, precision)


def dequantize_levels(symbols, outliers, counts, widths, precision="f64"):
    """Inverse of :func:`quantize_levels`: per-level coefficient vectors."""
    out = []
    pos = 0
    opos = 0
    for n, w in zip(counts, widths):
        s = symbols[pos:pos + n].astype(np.int64)
        esc = s == ESC
        ne = int(esc.sum())
        q = s - R
        if precision == "f32":
            c = (q.astype(np.float32) * np.float32(w)).astype(np.float32)
            qo = outliers[opos:opos + ne].astype(np.int64)
            small = np.abs(qo) < F32_EXACT
            c[esc] = np.where(small, qo.astype(np.float32) * np.float32(w),
                              (qo.astype(np.float64) * w).astype(np.float32))
        else:
            c = q.astype(np.float64) * w
            c[esc] = outliers[opos:opos + ne].astype(np.float64) * w
        out.append(c)
        pos += n
        opos += ne
    return out


def level_counts(shape, max_levels=None):
    h = hierarchy(shape, max_levels)
    if h.D == 0:
        return [1]
    return [h.new_count(l) for l in range(h.L + 1)]


def scatter_levels(levels, shape, max_levels=None):
    """Place per-level coefficient vectors back into the in-place layout
    (inverse of :func:`multilevel.level_coefficients`)."""
    h = hierarchy(shape, max_levels)
    if h.D == 0:
        return np.asarray(levels[0], dtype=np.float64).reshape(shape)
    out = np.zeros(h.squeezed, dtype=np.float64)
    for l in range(h.L + 1):
        sub = np.ix_(*h.idx[l])
        U = out[sub]
        if l == 0:
            U[...] = np.asarray(levels[0], dtype=np.float64).reshape(U.shape)
        else:
            mask = np.ones(U.shape, dtype=bool)
            mask[np.ix_(*[h.coarse_pos(l, d) for d in range(h.D)])] = False
            U[mask] = levels[l]
        out[sub] = U
    return out.reshape(h.shape)
