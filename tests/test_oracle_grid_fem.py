"""Pins for the oracle's hierarchy and 1D finite-element operators."""
import itertools

import numpy as np
import pytest
import sympy

from oracle import fem, grid


@pytest.mark.parametrize("m,expect", [
    (3, [0, 2]), (4, [0, 2, 3]), (5, [0, 2, 4]), (6, [0, 2, 4, 5]), (7, [0, 2, 4, 6]),
])
def test_coarse_positions_even_plus_last(m, expect):
    assert grid.coarse_positions(m).tolist() == expect


@pytest.mark.parametrize("n,L", [(2, 0), (3, 1), (4, 2), (5, 2), (129, 7), (513, 9),
                                 (1025, 10), (256, 8), (384, 9), (33, 5), (65, 6),
                                 (257, 8), (300, 9)])
def test_axis_levels(n, L):
    assert grid.axis_levels(n) == L


def test_hierarchy_min_levels_and_squeeze():
    h = grid.hierarchy((1, 33, 1, 300))
    assert h.squeezed == (33, 300) and h.L == 5
    assert grid.hierarchy((7, 2)).L == 0
    assert grid.hierarchy((1, 1)).D == 0
    assert grid.hierarchy((513, 513, 513), max_levels=3).L == 3


def test_node_level_is_first_appearance():
    h = grid.hierarchy((9, 6, 7))
    lev = grid.node_level(h)
    sets = [set(itertools.product(*[a.tolist() for a in h.idx[l]])) for l in range(h.L + 1)]
    for node in itertools.product(*[range(n) for n in h.squeezed]):
        first = min(l for l in range(h.L + 1) if node in sets[l])
        assert lev[node] == first


def _sym_hat(xs, j, x):
    """Exact hat function j on nodes xs as a sympy Piecewise."""
    pieces = []
    if j > 0:
        a, b = xs[j - 1], xs[j]
        pieces.append(((x - a) / (b - a), (x >= a) & (x <= b)))
    if j < len(xs) - 1:
        a, b = xs[j], xs[j + 1]
        pieces.append(((b - x) / (b - a), (x >= a) & (x <= b)))
    pieces.append((0, True))
    return sympy.Piecewise(*pieces)


def test_mass_matrix_matches_symbolic_integration():
    xs = [sympy.Integer(v) for v in (0, 2, 3, 7, 8)]
    x = sympy.Symbol("x", real=True)
    M = fem.mass_matrix(np.array([float(v) for v in xs])).toarray()
    for i in range(len(xs)):
        for j in range(len(xs)):
            # integrate piecewise over each element where both hats live
            val = 0
            for e in range(len(xs) - 1):
                a, b = xs[e], xs[e + 1]
                hi = sympy.piecewise_fold(_sym_hat(xs, i, x) * _sym_hat(xs, j, x))
                val += sympy.integrate(hi, (x, a, b))
            assert abs(M[i, j] - float(val)) < 1e-14


def test_prolongation_reproduces_linears_and_partition_of_unity():
    xf = np.array([0., 1., 2., 3., 4., 5.])
    xc = xf[grid.coarse_positions(6)]
    P = fem.prolongation(xf, xc).toarray()
    assert np.allclose(P.sum(axis=1), 1.0)
    assert np.allclose(P @ (3 * xc - 1), 3 * xf - 1)
    # non-uniform: coarse {0, 4, 5}, fine node 4 between 0 and 5 is not new here,
    # but node at 2 between 0 and 4 gets weights 1/2, 1/2
    P2 = fem.prolongation(np.array([0., 2., 4., 5.]), np.array([0., 4., 5.])).toarray()
    assert np.allclose(P2[1], [0.5, 0.5, 0.0])
    P3 = fem.prolongation(np.array([0., 4., 5.]), np.array([0., 5.])).toarray()
    assert np.allclose(P3[1], [0.2, 0.8])


def test_banded_equals_sparse_mass():
    x = np.array([0., 1., 3., 4., 9.])
    ab = fem.mass_banded(x)
    M = fem.mass_matrix(x).toarray()
    rebuilt = np.diag(ab[1]) + np.diag(ab[0, 1:], 1) + np.diag(ab[2, :-1], -1)
    assert np.allclose(rebuilt, M)
