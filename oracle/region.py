"""Region-adaptive L-infinity error bounds (oracle; test infrastructure).

The paper ("Application impact", Earth and cosmological science) describes
compression that keeps a tighter error in chosen regions of a field than
elsewhere (spatially adaptive compression of climate output); it prints no
method.  The reading used here is rigorous, in FP64:

Request   a background absolute tolerance ``tau`` and boxes ``B_r``
          (inclusive index ranges per axis of the input grid) with
          tolerances ``tau_r <= tau``.  Guarantee: ``|u~(p) - u(p)|`` is at
          most the smallest ``tau_r`` of the boxes holding ``p``, and at most
          ``tau`` everywhere.

Error of the recomposition.  With ``dz_l`` the errors of the level-l
coefficients, ``C_l = M_{l-1}^{-1} P^T M_l`` the correction operator and
``Pi`` interpolation, one recomposition step gives
``e_l = Pi(e_{l-1} - C_l dz_l) + dz_l``, so the error at a node ``p`` of the
input grid is a sum over levels of interpolated values.  Interpolation
takes convex combinations of the corners of the cell around ``p``, so level
``l`` contributes at most ``max_q |dz_l(q)| + max_j sum_i |C_l(j, i)| |dz_l(i)|``
over the level-l corners ``q`` of ``p``'s cell and the level-(l-1) corners
``j`` of ``q``'s cell.  ``C_l`` is the tensor product of 1D operators whose
entries decay geometrically away from the coarse node, so the sum splits
into the entries within ``rho`` level-l nodes of ``j`` on every axis, which
see the small widths of the region, and a far-field tail weighted by the
background width:

* ``S_{l,d}``: the row-sum norm of the axis operator (their product is
  ``K_l``);
* ``t_{l,d}(rho)``: the largest row sum of the entries more than ``rho``
  level-l nodes from the row's coarse node;
* ``T_l(rho) = sum_d t_{l,d}(rho) prod_{e != d} S_{l,e}`` bounds the tail of
  the tensor operator (the difference of two products, telescoped).

Rule
    ``den = 1 + sum_l c_l``, the constant of the uniform L-infinity width
    (``c_l`` bounds the row sums of level l's whole error operator, so also
    the part of a row inside the dilation), and ``w_bg = 2 tau / den`` that
    width (with the compressor's margin).
    ``rho``: the smallest radius in ``0 .. RHO_MAX`` with
    ``tau sum_l T_l(rho) / den <= min_r tau_r / 8``.
    ``k_r``: the smallest ``k >= 0`` with
    ``2^-k tau <= tau_r - tau sum_l T_l(rho) / den``.
    Dilation of a box on level l along axis d: ``m_{0,d} = H_{0,d}`` and
    ``m_{l,d} = (rho + 1) H_{l,d} + H_{l-1,d}`` with ``H_{l,d}`` the largest
    spacing of the level-l nodes on that axis (input-grid units).
    A node first appearing on level l gets the width ``w_bg 2^-k`` with
    ``k`` the largest ``k_r`` of the boxes whose dilation contains it (0 if
    none).  Every node near enough to reach a point of ``B_r`` through the
    corners and the first ``rho`` entries of ``C_l`` is inside the dilation,
    so at a point of ``B_r`` the error is at most
    ``(w_bg 2^-k_r / 2) den + (w_bg / 2) sum_l T_l(rho) <= tau_r``.
Widths are powers of two below the background width, so scaling a
coefficient by ``2^k`` and quantizing it with ``w_bg`` gives the same
integer as quantizing it with ``w_bg 2^-k``.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

from . import bounds, fem, multilevel
from .grid import hierarchy, node_level

RHO_MAX = 48


def axis_operator(h, l: int, d: int) -> np.ndarray:
    """Dense 1D correction operator ``M_c^{-1} P^T M_f`` of level l on axis d."""
    xf, xc = h.coords(l, d), h.coords(l - 1, d)
    P = fem.prolongation(xf, xc).toarray()
    Mf = fem.mass_matrix(xf).toarray()
    Mc = fem.mass_matrix(xc).toarray()
    return scipy.linalg.solve(Mc, P.T @ Mf)


def axis_norm_and_tails(h, l: int, d: int):
    """(S, t[0..RHO_MAX]) of the level-l operator on axis d."""
    C = np.abs(axis_operator(h, l, d))
    pos = h.coarse_pos(l, d)
    S = float(np.max(C.sum(axis=1)))
    i = np.arange(C.shape[1])
    t = np.empty(RHO_MAX + 1)
    for rho in range(RHO_MAX + 1):
        far = np.abs(i[None, :] - pos[:, None]) > rho
        t[rho] = float(np.max(np.where(far, C, 0.0).sum(axis=1)))
    return S, t


def tail_bounds(h, l: int) -> np.ndarray:
    """``T_l(rho)`` for rho = 0..RHO_MAX."""
    St = [axis_norm_and_tails(h, l, d) for d in range(h.D)]
    T = np.zeros(RHO_MAX + 1)
    for d in range(h.D):
        other = 1.0
        for e in range(h.D):
            if e != d:
                other *= St[e][0]
        T += St[d][1] * other
    return T


def max_spacing(h, l: int, d: int) -> int:
    x = h.idx[l][d]
    return int(np.max(np.diff(x))) if len(x) > 1 else 0


def _squeeze_box(shape, lo, hi):
    keep = [a for a, n in enumerate(shape) if n > 1]
    return [int(lo[a]) for a in keep], [int(hi[a]) for a in keep]


def plan(shape, tol: float, regions):
    """Radius, per-region exponents and per-level dilated boxes.

    ``regions``: list of ``(lo, hi, tol_r)`` with ``lo``/``hi`` index tuples
    of the input shape (inclusive)."""
    h = hierarchy(shape)
    if h.L < 1:
        raise ValueError("regions need at least one level")
    den = bounds.linf_denominator(h)
    T = [tail_bounds(h, l) for l in range(1, h.L + 1)]
    tmin = min([r[2] for r in regions] + [tol])
    rho = None
    for c in range(RHO_MAX + 1):
        if tol * sum(t[c] for t in T) / den <= tmin / 8.0:
            rho = c
            break
    if rho is None:
        raise ValueError("region tolerances too small against the background")
    far = tol * sum(t[rho] for t in T) / den
    ks = []
    for (_, _, tr) in regions:
        if not (0.0 < tr <= tol):
            raise ValueError("a region's tolerance must lie in (0, tol]")
        k = 0
        while math.ldexp(tol, -k) > tr - far:
            k += 1
        ks.append(k)
    H = [[max_spacing(h, l, d) for d in range(h.D)] for l in range(h.L + 1)]
    margins = [[H[0][d] for d in range(h.D)]]
    for l in range(1, h.L + 1):
        margins.append([(rho + 1) * H[l][d] + H[l - 1][d] for d in range(h.D)])
    boxes = []
    for (lo, hi, _) in regions:
        slo, shi = _squeeze_box(shape, lo, hi)
        boxes.append([[(slo[d] - margins[l][d], shi[d] + margins[l][d]) for d in range(h.D)]
                      for l in range(h.L + 1)])
    return dict(rho=rho, k=ks, margins=margins, boxes=boxes, far=far, den=den,
                w_bg=float(bounds.bin_widths(shape, tol, math.inf)[0]))


def exponents(shape, tol: float, regions) -> np.ndarray:
    """Width exponent ``k`` of every node of the input grid."""
    pl = plan(shape, tol, regions)
    h = hierarchy(shape)
    lev = node_level(h).reshape(h.squeezed)
    k = np.zeros(h.squeezed, dtype=np.int64)
    grids = np.meshgrid(*[np.arange(n) for n in h.squeezed], indexing="ij")
    for r, kr in enumerate(pl["k"]):
        for l in range(h.L + 1):
            inside = lev == l
            for d in range(h.D):
                a, b = pl["boxes"][r][l][d]
                inside &= (grids[d] >= a) & (grids[d] <= b)
            k = np.where(inside, np.maximum(k, kr), k)
    return k.reshape(shape)


def node_widths(shape, tol: float, regions) -> np.ndarray:
    pl = plan(shape, tol, regions)
    return np.ldexp(pl["w_bg"], -exponents(shape, tol, regions))


def compress(u: np.ndarray, tol: float, regions):
    """Decompose and quantize every coefficient with its node's width (FP64,
    round half to even); returns the integers and the widths."""
    w = node_widths(u.shape, tol, regions)
    v = multilevel.decompose(u)
    return np.rint(v / w), w


def decompress(q: np.ndarray, w: np.ndarray) -> np.ndarray:
    return multilevel.recompose(q * w)


def tolerance_map(shape, tol: float, regions) -> np.ndarray:
    """The guaranteed bound at every node: min of the tolerances of the boxes
    that hold it, tol elsewhere."""
    t = np.full(shape, float(tol))
    for lo, hi, tr in regions:
        sl = tuple(slice(a, b + 1) for a, b in zip(lo, hi))
        t[sl] = np.minimum(t[sl], tr)
    return t
