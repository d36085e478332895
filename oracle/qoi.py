"""Error control of linear quantities of interest (oracle; test infrastructure).

The paper ("Software design"; "Application impact", plasma physics) says
MGARD guarantees the error of quantities of interest (QoIs) derived from the
data, not only the error of the data, and prints no formula.  The reading
used here, for linear QoIs, in FP64:

QoI          ``Q(v) = sum_p g_p v_p`` with weights ``g`` on the nodes of the
             input grid (a region average, a weighted sum, a point value).
Representer  the P1 function ``r`` in ``V_L`` with ``<r, v>_{L2} = Q(v)`` for
             every ``v`` in ``V_L``: ``M_L r = g`` with ``M_L`` the tensor
             product of the 1D mass matrices, i.e. one tridiagonal solve
             along each axis.
Dual norm    ``||Q||_{-s} = ||r||_{-s}``: the s-norm with ``-s`` in place of
             ``s``.  ``V_L`` is the orthogonal sum of the ranges of
             ``Q_l - Q_{l-1}``, so with ``r_l, e_l`` the components,
             ``Q(e) = sum_l <r_l, e_l> <= sum_l 2^{-sl}|r_l| 2^{sl}|e_l|
             <= ||r||_{-s} ||e||_s`` (Cauchy-Schwarz in each term and then
             over the levels).  For ``s = inf`` (nodal maximum norm):
             ``|Q(e)| <= ||g||_1 max|e|``.
Control      a QoI tolerance ``tau_Q`` becomes the absolute s-norm tolerance
             ``tau_Q / ||Q||_{-s}``; the compressor's guarantee
             ``||e||_s <= tol`` then gives ``|Q(u~) - Q(u)| <= tau_Q``.
"""
from __future__ import annotations

import math

import numpy as np

from . import bounds, fem, pipeline
from .grid import hierarchy


def representer(g: np.ndarray, max_levels=None) -> np.ndarray:
    """``r = M_L^{-1} g`` on the input grid (FP64, the shape of ``g``)."""
    g = np.asarray(g, dtype=np.float64)
    h = hierarchy(g.shape, max_levels)
    if h.D == 0:
        return g.copy()
    R = g.reshape(h.squeezed)
    for d in range(h.D):
        R = fem.solve_along(fem.mass_banded(h.coords(h.L, d)), R, d)
    return R.reshape(g.shape)


def norm(g: np.ndarray, s: float, max_levels=None) -> float:
    """``||Q||_{-s}`` of the QoI with weights ``g`` (``||g||_1`` for s = inf)."""
    if math.isinf(s):
        return float(np.sum(np.abs(np.asarray(g, dtype=np.float64))))
    return bounds.s_norm(representer(g, max_levels), -s, max_levels)


def value(u: np.ndarray, g: np.ndarray) -> float:
    """``Q(u) = sum_p g_p u_p`` (FP64)."""
    return float(np.sum(np.asarray(g, dtype=np.float64) * np.asarray(u, dtype=np.float64)))


def tolerance(g: np.ndarray, tol_qoi: float, s: float, max_levels=None) -> float:
    """Absolute s-norm tolerance that keeps ``|Q(u~) - Q(u)| <= tol_qoi``."""
    return tol_qoi / norm(g, s, max_levels)


def compress(u: np.ndarray, g: np.ndarray, tol_qoi: float, s: float, max_levels=None):
    """Compress ``u`` so that the QoI's error stays within ``tol_qoi``."""
    return pipeline.compress(u, tolerance(g, tol_qoi, s, max_levels), s, relative=False,
                             max_levels=max_levels)
