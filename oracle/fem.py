"""1D piecewise-linear finite-element operators (oracle; test infrastructure).

The paper attributes MGARD's error guarantee to finite element theory
("Motivation and significance", last paragraphs; "Software design").  The
standard P1 definitions used by the decomposition are written out here on a
level's node coordinates ``x_0 < ... < x_{m-1}`` with spacings
``h_i = x_{i+1} - x_i``:

* hat function ``phi_i``: 1 at ``x_i``, 0 at every other node, linear between;
* mass matrix ``M_ij = integral phi_i phi_j`` (exact for hats):
  ``M_ii = (h_{i-1} + h_i) / 3``, ``M_{i,i+1} = M_{i+1,i} = h_i / 6``
  (with ``h_{-1} = h_{m-1} = 0``);
* prolongation ``P`` (coarse -> fine): ``P_ij`` = coarse hat ``j`` evaluated at
  fine node ``i`` (so ``P`` is linear interpolation of coarse nodal values).

Multi-dimensional operators are tensor products of these; ``apply_along``
applies a 1D operator to one axis of an array.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp


def mass_matrix(x: np.ndarray) -> sp.csr_matrix:
    x = np.asarray(x, dtype=np.float64)
    m = len(x)
    h = np.diff(x)
    diag = np.zeros(m)
    diag[:-1] += h / 3.0
    diag[1:] += h / 3.0
    off = h / 6.0
    return sp.diags([off, diag, off], [-1, 0, 1], shape=(m, m), format="csr")


def mass_banded(x: np.ndarray) -> np.ndarray:
    """The same tridiagonal mass matrix in LAPACK banded storage (3 x m)."""
    x = np.asarray(x, dtype=np.float64)
    m = len(x)
    h = np.diff(x)
    ab = np.zeros((3, m))
    ab[0, 1:] = h / 6.0
    ab[1, :-1] += h / 3.0
    ab[1, 1:] += h / 3.0
    ab[2, :-1] = h / 6.0
    return ab


def prolongation(xf: np.ndarray, xc: np.ndarray) -> sp.csr_matrix:
    """Interpolation from coarse nodes ``xc`` (a subset of ``xf``) to ``xf``."""
    xf = np.asarray(xf, dtype=np.float64)
    xc = np.asarray(xc, dtype=np.float64)
    rows, cols, vals = [], [], []
    for i, x in enumerate(xf):
        j = int(np.searchsorted(xc, x))
        if j < len(xc) and xc[j] == x:
            rows.append(i); cols.append(j); vals.append(1.0)
            continue
        a, b = xc[j - 1], xc[j]
        rows += [i, i]
        cols += [j - 1, j]
        vals += [(b - x) / (b - a), (x - a) / (b - a)]
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(xf), len(xc)))


def apply_along(A, X: np.ndarray, axis: int) -> np.ndarray:
    """Return ``X`` with the linear map ``A`` (rows x len) applied along ``axis``."""
    Xm = np.moveaxis(X, axis, 0)
    shp = Xm.shape
    Y = A @ Xm.reshape(shp[0], -1)
    Y = np.asarray(Y).reshape((A.shape[0],) + shp[1:])
    return np.moveaxis(Y, 0, axis)


def solve_along(ab: np.ndarray, X: np.ndarray, axis: int) -> np.ndarray:
    """Solve the tridiagonal system (banded storage ``ab``) along ``axis``."""
    Xm = np.moveaxis(X, axis, 0)
    shp = Xm.shape
    Y = scipy.linalg.solve_banded((1, 1), ab, Xm.reshape(shp[0], -1))
    return np.moveaxis(Y.reshape(shp), 0, axis)
