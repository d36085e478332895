"""Multilevel decomposition and recomposition (oracle; test infrastructure).

Follows the paper's "Software design" section: the data ``u`` is decomposed
recursively into multilevel coefficients ``u_mc`` on the grid hierarchy, and
recomposition is the inverse procedure.  With ``V_l`` the tensor-product P1
space on the level-l nodes, ``Q_l`` the L2 projection onto ``V_l`` and
``Pi_l`` nodal interpolation onto ``V_l``, one step l -> l-1 of the
decomposition is written out as:

1. interpolation coefficients: ``z = u_l - Pi_{l-1} u_l`` (zero on the coarse
   nodes; its values on the new nodes are the level-l coefficients);
2. load vector: ``b = P^T M_l z`` (mass matrix, then restriction), one axis at
   a time;
3. coarse solve: ``M_{l-1} c = b``, a tridiagonal solve along each axis;
4. correction: ``u_{l-1} = u_l|coarse + c``, the nodal values of
   ``Q_{l-1} u_l``.

The result is stored in place: each node keeps the coefficient of the level
on which it first appears; level-0 nodes keep the values of ``Q_0 u``.
Everything is FP64.
"""
from __future__ import annotations

import numpy as np

from . import fem
from .grid import Hierarchy, hierarchy


def _tensor(ops, X):
    for d, A in enumerate(ops):
        X = fem.apply_along(A, X, d)
    return X


def _tensor_solve(abs_, X):
    for d, ab in enumerate(abs_):
        X = fem.solve_along(ab, X, d)
    return X


def _level_ops(h: Hierarchy, l: int):
    """1D operators for the step between level l and l-1 on every axis."""
    P, Mf, Mc_ab = [], [], []
    for d in range(h.D):
        xf = h.coords(l, d)
        xc = h.coords(l - 1, d)
        P.append(fem.prolongation(xf, xc))
        Mf.append(fem.mass_matrix(xf))
        Mc_ab.append(fem.mass_banded(xc))
    return P, Mf, Mc_ab


def correction(h: Hierarchy, l: int, z: np.ndarray) -> np.ndarray:
    """Coarse-grid correction ``M_{l-1}^{-1} P^T M_l z`` for a level-l array ``z``."""
    P, Mf, Mc_ab = _level_ops(h, l)
    f = _tensor(Mf, z)                              # f = M_l z
    b = _tensor([p.T.tocsr() for p in P], f)        # b = P^T f
    return _tensor_solve(Mc_ab, b)                  # M_{l-1} c = b


def interpolate(h: Hierarchy, l: int, uc: np.ndarray) -> np.ndarray:
    """Multilinear interpolation of level-(l-1) nodal values onto level l."""
    P, _, _ = _level_ops(h, l)
    return _tensor(P, uc)


def decompose(u: np.ndarray, max_levels=None) -> np.ndarray:
    """Multilevel coefficients of ``u`` in the in-place layout (FP64)."""
    h = hierarchy(u.shape, max_levels)
    v = np.array(u, dtype=np.float64).reshape(h.squeezed if h.D else (1,))
    for l in range(h.L, 0, -1):
        fine = np.ix_(*h.idx[l])
        cpos = np.ix_(*[h.coarse_pos(l, d) for d in range(h.D)])
        U = v[fine]
        Uc = U[cpos]
        z = U - interpolate(h, l, Uc)               # step 1
        corr = correction(h, l, z)                  # steps 2-3
        z[cpos] = Uc + corr                         # step 4 (coarse nodes)
        v[fine] = z
    return v.reshape(h.shape)


def recompose(v: np.ndarray, max_levels=None) -> np.ndarray:
    """Inverse of :func:`decompose`."""
    h = hierarchy(v.shape, max_levels)
    u = np.array(v, dtype=np.float64).reshape(h.squeezed if h.D else (1,))
    for l in range(1, h.L + 1):
        fine = np.ix_(*h.idx[l])
        cpos = np.ix_(*[h.coarse_pos(l, d) for d in range(h.D)])
        U = u[fine]
        proj = U[cpos].copy()                       # nodal values of Q_{l-1} u
        z = U.copy()
        z[cpos] = 0.0                               # coefficient function z
        Uc = proj - correction(h, l, z)             # coarse values of u_l
        U = interpolate(h, l, Uc) + z               # u_l = Pi u_l + z
        u[fine] = U
    return u.reshape(h.shape)


def projections(u: np.ndarray, max_levels=None):
    """Nodal values of ``Q_l u`` on every level (list indexed by l)."""
    h = hierarchy(u.shape, max_levels)
    v = np.array(u, dtype=np.float64).reshape(h.squeezed if h.D else (1,))
    out = [None] * (h.L + 1)
    U = v
    out[h.L] = U.copy()
    for l in range(h.L, 0, -1):
        cpos = np.ix_(*[h.coarse_pos(l, d) for d in range(h.D)])
        Uc = U[cpos]
        z = U - interpolate(h, l, Uc)
        U = Uc + correction(h, l, z)
        out[l - 1] = U.copy()
    return out


def mass_norm2(h: Hierarchy, l: int, U: np.ndarray) -> float:
    """``U^T M_l U``: squared L2 norm of the level-l P1 function with nodal
    values ``U``."""
    M = [fem.mass_matrix(h.coords(l, d)) for d in range(h.D)]
    return float(np.sum(U * _tensor(M, U)))


def level_coefficients(v: np.ndarray, max_levels=None):
    """Split an in-place decomposed array into per-level flat coefficient
    vectors in row-major order of each level's grid (new nodes only; level 0
    holds all its nodes)."""
    h = hierarchy(v.shape, max_levels)
    a = np.asarray(v).reshape(h.squeezed if h.D else (1,))
    out = []
    for l in range(h.L + 1):
        U = a[np.ix_(*h.idx[l])] if h.D else a
        if l == 0:
            out.append(U.reshape(-1).copy())
            continue
        mask = np.ones(U.shape, dtype=bool)
        mask[np.ix_(*[h.coarse_pos(l, d) for d in range(h.D)])] = False
        out.append(U[mask].copy())
    return out
