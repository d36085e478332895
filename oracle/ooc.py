"""Out-of-core blocking (oracle; test infrastructure).

The paper ("Software architecture") names an out-of-core module that cuts
arrays too large for device memory into pieces compressed one by one.  The
reading used here: the field is cut along its first axis into ``nblocks``
blocks of as equal sizes as possible (the first ``n0 % nblocks`` blocks one
index plane larger), every block is compressed on its own hierarchy with the
L-infinity bound (absolute; a relative tolerance is scaled by max|u| of the
whole field), and the reconstruction is the blocks' reconstructions side by
side.  Every node lies in exactly one block, so the whole field keeps the
bound.
"""
from __future__ import annotations

import math

import numpy as np

from . import pipeline


def block_ranges(n0: int, nblocks: int):
    """[(begin, end)) of every block along the first axis."""
    if not 1 <= nblocks <= n0:
        raise ValueError("1 <= nblocks <= n0")
    q, r = divmod(n0, nblocks)
    out, b0 = [], 0
    for b in range(nblocks):
        n = q + (1 if b < r else 0)
        out.append((b0, b0 + n))
        b0 += n
    return out


def tolerance(u: np.ndarray, tol: float, relative: bool) -> float:
    return tol * float(np.max(np.abs(np.asarray(u, dtype=np.float64)))) if relative else tol


def compress(u: np.ndarray, tol: float, nblocks: int, relative: bool = False):
    tol_abs = tolerance(u, tol, relative)
    return [pipeline.compress(u[a:b], tol_abs, math.inf, relative=False)
            for a, b in block_ranges(u.shape[0], nblocks)], tol_abs


def decompress(blocks) -> np.ndarray:
    return np.concatenate([pipeline.decompress(c) for c in blocks], axis=0)
