"""Node hierarchy of a structured grid (oracle; test infrastructure only).

The paper's "Software design" section decomposes the data "over a multigrid
hierarchy" of a structured grid without fixing how non-dyadic sizes coarsen.
Readings used here:

* Axis order is row-major (last axis contiguous).  Axes of extent 1 are
  squeezed out before anything else.
* Coordinates are the finest-grid indices (spacing 1 on the input grid).
* Along one axis, the nodes of the next coarser level are the even positions
  of the current level plus its last position (so both ends are kept and a
  level of ``m`` nodes has ``m // 2 + 1`` coarse nodes).  Coarsening stops at
  two nodes.
* The level count is ``L = min_d L_d`` where ``L_d`` is the number of
  coarsenings axis ``d`` allows; every axis coarsens at every level.  An
  optional ``max_levels`` caps ``L``.  Level ``L`` is the input grid, level 0
  the coarsest.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def coarse_positions(m: int) -> np.ndarray:
    """Positions, within a level of ``m >= 3`` nodes, of the nodes kept on the
    next coarser level: every even position plus the last one."""
    pos = list(range(0, m, 2))
    if pos[-1] != m - 1:
        pos.append(m - 1)
    return np.asarray(pos, dtype=np.int64)


def axis_levels(n: int) -> int:
    """How many times an axis of ``n >= 2`` nodes can coarsen before it has
    two nodes."""
    count = 0
    m = n
    while m > 2:
        m = len(coarse_positions(m))
        count += 1
    return count


@dataclass
class Hierarchy:
    shape: tuple            # original shape
    squeezed: tuple         # shape with extent-1 axes removed
    L: int                  # number of levels above level 0
    idx: list               # idx[l][d]: finest-grid indices of level-l nodes on axis d

    @property
    def D(self) -> int:
        return len(self.squeezed)

    def level_shape(self, l: int) -> tuple:
        return tuple(len(a) for a in self.idx[l])

    def coords(self, l: int, d: int) -> np.ndarray:
        return self.idx[l][d].astype(np.float64)

    def coarse_pos(self, l: int, d: int) -> np.ndarray:
        """Positions of level-(l-1) nodes inside the level-l node list."""
        return np.searchsorted(self.idx[l][d], self.idx[l - 1][d])

    def new_count(self, l: int) -> int:
        """Number of nodes first appearing on level l (all nodes for l=0)."""
        n = int(np.prod(self.level_shape(l)))
        if l == 0:
            return n
        return n - int(np.prod(self.level_shape(l - 1)))


def hierarchy(shape, max_levels=None) -> Hierarchy:
    shape = tuple(int(s) for s in shape)
    if len(shape) < 1 or len(shape) > 4 or any(s < 1 for s in shape):
        raise ValueError("shape must have 1..4 positive extents")
    squeezed = tuple(s for s in shape if s > 1)
    if not squeezed:
        return Hierarchy(shape, squeezed, 0, [[]])
    L = min(axis_levels(n) for n in squeezed)
    if max_levels is not None and max_levels >= 0:
        L = min(L, int(max_levels))
    idx = [None] * (L + 1)
    idx[L] = [np.arange(n, dtype=np.int64) for n in squeezed]
    for l in range(L, 0, -1):
        idx[l - 1] = [a[coarse_positions(len(a))] for a in idx[l]]
    return Hierarchy(shape, squeezed, L, idx)


def node_level(h: Hierarchy) -> np.ndarray:
    """Level at which each node of the input grid first appears: the maximum
    over axes of the level at which its index on that axis first appears."""
    if h.D == 0:
        return np.zeros(h.shape, dtype=np.int64)
    per_axis = []
    for d, n in enumerate(h.squeezed):
        lv = np.full(n, h.L, dtype=np.int64)
        for l in range(h.L - 1, -1, -1):
            lv[h.idx[l][d]] = l
        per_axis.append(lv)
    grids = np.meshgrid(*per_axis, indexing="ij")
    out = grids[0]
    for g in grids[1:]:
        out = np.maximum(out, g)
    return out
