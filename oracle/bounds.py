"""Error estimators: bin widths and error norms (oracle; test infrastructure).

The paper ("Software design") says compression quantizes every multilevel
coefficient to a multiple of a bin width, that the widths come from error
estimators taking the quantization errors as inputs, and that the bound is
guaranteed in several norms selected by the smoothness parameter ``s``.  It
gives no constants.  The widths below are derived here from the P1
definitions (readings, listed in full in the design notes):

L-infinity (``s = inf``)
    Recomposition of quantization errors ``delta_l`` (|delta_l| <= w/2) adds
    at level l, on the level-l grid, ``A_l delta_l`` with
    ``A_l = I_new - P C_l`` (``C_l = M_{l-1}^{-1} P^T M_l`` the correction
    operator, ``P`` interpolation from level l-1, ``I_new`` the identity on
    the new nodes; the coarse nodes carry no coefficient), and finer levels
    only interpolate it (convex combinations).  So
    ``||e||_inf <= (w/2) (1 + sum_{l>=1} c_l)`` with ``c_l`` the largest
    row sum ``max_q sum_{i new} |A_l(q, i)|``.  ``P C_l`` is the tensor
    product of the axis matrices ``B_d = P_d C_d``, so with, per axis and
    row, ``T = sum_i |B(q, i)|``, ``Tc`` the same over coarse columns and
    ``b = B(q, q)``:
    ``sum_{i new} |A(q, i)| = prod T - prod Tc + [q new] (|1 - prod b| - prod |b|)``.
    ``c_l`` bounds its maximum by splitting the rows by which axes are
    coarse (2^D classes) and taking, per axis and class, the largest ``T``,
    the smallest ``Tc``, the range of ``b`` and the smallest ``|b|``.  One
    width for every level: ``w = 2 tau / (1 + sum_l c_l)``.  (An earlier,
    looser reading bounded each row by ``1 + K_l`` with
    ``K_l = prod_d ||C_d||_inf``; ``K_l`` is kept for the refactoring
    estimate and the region bounds.)

s-norm (finite ``s >= 0``)
    ``||e||_s^2 = sum_{l=0..L} 4^{s l} ||(Q_l - Q_{l-1}) e||^2`` (``Q_{-1} = 0``;
    ``s = 0`` is the L2 norm by orthogonality).  The level-l term is at most
    ``delta_l^T M_l delta_l <= mu_l ||delta_l||_2^2`` with the Gershgorin bound
    ``mu_l = prod_d max_i (h_{i-1} + h_i) / 2``, so
    ``w_l = 2 tau / sqrt((L + 1) 4^{s l} mu_l n_l)`` with ``n_l`` the number
    of new nodes on level l.

Every width is then multiplied by ``1 - 2^-8``.  That margin absorbs the
rounding of a single-precision quantizer (``x = c * (1/w)`` and ``q * w``
each rounded to float32 for ``|q| < 4096``: at most 0.5 + 4096.5 * 2^-23
bins for ``q`` plus 4096 * 2^-23 bins for the product, which the margin
brings back under half of the unscaled width), so ``|c - q w| <= w_bound / 2``
holds for it too.

Relative tolerances scale by ``max|u|`` (L-infinity) or ``||u||_s``.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import fem
from .grid import Hierarchy, hierarchy
from .multilevel import mass_norm2, projections

WIDTH_MARGIN = 1.0 - 2.0 ** -8


def correction_norm_1d(h: Hierarchy, l: int, d: int) -> float:
    """``||(M_{l-1})^{-1} P^T M_l||_inf`` on axis d (dense, exact in FP64)."""
    xf, xc = h.coords(l, d), h.coords(l - 1, d)
    P = fem.prolongation(xf, xc).toarray()
    Mf = fem.mass_matrix(xf).toarray()
    Mc = fem.mass_matrix(xc).toarray()
    A = np.linalg.solve(Mc, P.T @ Mf)
    return float(np.abs(A).sum(axis=1).max())


def K(h: Hierarchy, l: int) -> float:
    k = 1.0
    for d in range(h.D):
        k *= correction_norm_1d(h, l, d)
    return k


def axis_level_rows(h: Hierarchy, l: int, d: int):
    """Per row q of ``B = P_d C_d`` on axis d (level-l grid): ``T``, ``Tc``,
    ``b`` and whether q is a coarse node (dense, FP64)."""
    xf, xc = h.coords(l, d), h.coords(l - 1, d)
    P = fem.prolongation(xf, xc).toarray()
    C = np.linalg.solve(fem.mass_matrix(xc).toarray(), P.T @ fem.mass_matrix(xf).toarray())
    B = P @ C
    coarse = np.zeros(len(xf), dtype=bool)
    coarse[h.coarse_pos(l, d)] = True
    A = np.abs(B)
    return A.sum(axis=1), A[:, coarse].sum(axis=1), np.diag(B).copy(), coarse


def linf_level_constant(h: Hierarchy, l: int) -> float:
    """``c_l``: an upper bound of ``max_q sum_{i new} |A_l(q, i)|`` from the
    per-axis class extremes (see the module docstring)."""
    rows = [axis_level_rows(h, l, d) for d in range(h.D)]
    best = 0.0
    for flags in itertools.product((True, False), repeat=h.D):   # True: coarse on that axis
        sel = [r[3] == f for r, f in zip(rows, flags)]
        if not all(np.any(x) for x in sel):
            continue
        t_max = 1.0
        tc_min = 1.0
        lo, hi = 1.0, 1.0        # range of prod b over the class (interval products)
        absb_min = 1.0
        for (T, Tc, b, _), x in zip(rows, sel):
            t_max *= float(np.max(T[x]))
            tc_min *= float(np.min(Tc[x]))
            bl, bh = float(np.min(b[x])), float(np.max(b[x]))
            cands = (lo * bl, lo * bh, hi * bl, hi * bh)
            lo, hi = min(cands), max(cands)
            absb_min *= float(np.min(np.abs(b[x])))
        v = t_max - tc_min
        if not all(flags):   # the class of new rows: the diagonal term
            v += max(abs(1.0 - lo), abs(1.0 - hi)) - absb_min
        best = max(best, v)
    return best


def linf_denominator(h: Hierarchy) -> float:
    """``1 + sum_l c_l``, summed in level order."""
    den = 1.0
    for l in range(1, h.L + 1):
        den += linf_level_constant(h, l)
    return den


def mu(h: Hierarchy, l: int) -> float:
    m = 1.0
    for d in range(h.D):
        x = h.coords(l, d)
        hh = np.diff(x)
        left = np.concatenate([[0.0], hh])
        right = np.concatenate([hh, [0.0]])
        m *= float(np.max((left + right) / 2.0))
    return m


def bin_widths(shape, tol_abs: float, s: float, max_levels=None) -> np.ndarray:
    """Quantization bin width of every level 0..L (FP64)."""
    h = hierarchy(shape, max_levels)
    L = h.L
    if math.isinf(s):
        w = np.full(L + 1, 2.0 * tol_abs / linf_denominator(h))
    else:
        w = np.empty(L + 1)
        for l in range(L + 1):
            m = mu(h, l) if h.D else 1.0
            n = h.new_count(l) if h.D else 1
            w[l] = 2.0 * tol_abs / math.sqrt((L + 1) * 4.0 ** (s * l) * m * n)
    return w * WIDTH_MARGIN


def s_norm(u: np.ndarray, s: float, max_levels=None) -> float:
    """``||u||_s`` from the projections ``Q_l u`` (FP64)."""
    h = hierarchy(u.shape, max_levels)
    if h.D == 0:
        return float(abs(np.asarray(u, dtype=np.float64).reshape(-1)[0]))
    Q = projections(u, max_levels)
    E = [mass_norm2(h, l, Q[l]) for l in range(h.L + 1)]
    total = E[0]
    for l in range(1, h.L + 1):
        total += 4.0 ** (s * l) * max(E[l] - E[l - 1], 0.0)
    return math.sqrt(max(total, 0.0))


def norm(u: np.ndarray, s: float, max_levels=None) -> float:
    if math.isinf(s):
        return float(np.max(np.abs(np.asarray(u, dtype=np.float64))))
    return s_norm(u, s, max_levels)
