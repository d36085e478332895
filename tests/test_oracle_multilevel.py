"""Pins for the oracle's decomposition: identities, exact special cases and a
brute-force dense L2 projection built by element quadrature (no tensor
factorization, no 1D operators from the oracle)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle import grid, multilevel

SHAPES = [(3,), (9,), (10,), (17, 17), (9, 6, 7), (5, 5, 5, 5), (33, 20), (1, 12, 1), (4, 13)]


@pytest.mark.parametrize("shape", SHAPES)
def test_recompose_inverts_decompose(shape):
    u = np.random.default_rng(1).standard_normal(shape)
    v = multilevel.decompose(u)
    r = multilevel.recompose(v)
    assert np.max(np.abs(r - u)) <= 1e-12 * max(1.0, np.max(np.abs(u)))


@pytest.mark.parametrize("shape", [(9,), (17, 9), (9, 6, 7), (5, 5, 5, 5), (7, 12)])
def test_multilinear_input_gives_zero_coefficients(shape):
    h = grid.hierarchy(shape)
    rng = np.random.default_rng(2)
    axes = [np.arange(n, dtype=float) for n in h.squeezed]
    X = np.meshgrid(*axes, indexing="ij")
    # a + sum b_d x_d + products of pairs: multilinear in each coordinate
    u = 0.7 + sum(rng.uniform(-1, 1) * x for x in X)
    for a, b in itertools.combinations(range(len(X)), 2):
        u = u + rng.uniform(-0.1, 0.1) * X[a] * X[b]
    v = multilevel.decompose(u)
    lev = grid.node_level(h)
    scale = np.max(np.abs(u))
    assert np.max(np.abs(v[lev > 0])) <= 1e-12 * scale
    # level-0 values are the samples themselves (Q_0 u = u for u in V_0)
    assert np.max(np.abs(v[lev == 0] - u[lev == 0])) <= 1e-12 * scale


def test_constant_input():
    u = np.full((9, 5, 6), 3.25)
    v = multilevel.decompose(u)
    lev = grid.node_level(grid.hierarchy(u.shape))
    assert np.max(np.abs(v[lev > 0])) < 1e-13
    assert np.allclose(v[lev == 0], 3.25)


def test_golden_1d_three_nodes():
    path = __file__.replace("test_oracle_multilevel.py", "golden/decompose_1d_n3.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        lhs, rhs = line.split("|")
        u = np.array([float(Fraction(t)) for t in lhs.split()])
        exp = np.array([float(Fraction(t)) for t in rhs.split()])
        assert np.allclose(multilevel.decompose(u), exp, atol=1e-15)


# --- brute-force dense projection -------------------------------------------

def _hat_eval(nodes, j, x):
    """Value at points x of the hat function of node j on a 1D node list."""
    x = np.asarray(x, dtype=float)
    out = np.zeros_like(x)
    if j > 0:
        a, b = nodes[j - 1], nodes[j]
        m = (x >= a) & (x <= b)
        out[m] = (x[m] - a) / (b - a)
    if j < len(nodes) - 1:
        a, b = nodes[j], nodes[j + 1]
        m = (x >= a) & (x <= b)
        out[m] = np.maximum(out[m], (b - x[m]) / (b - a))
    if len(nodes) == 1:
        out[:] = 1.0
    return out


def _gram(fine_nodes, left_nodes, right_nodes):
    """Gram matrix int phi_i psi_j over the tensor grid of ``fine_nodes``
    cells, by tensor Simpson quadrature on every cell (exact for products of
    multilinear functions); phi from ``left_nodes``, psi from ``right_nodes``."""
    D = len(fine_nodes)
    lsz = [len(a) for a in left_nodes]
    rsz = [len(a) for a in right_nodes]
    G = np.zeros((int(np.prod(lsz)), int(np.prod(rsz))))
    simpson = np.array([1.0, 4.0, 1.0]) / 6.0
    cells = [range(len(a) - 1) for a in fine_nodes]
    for cell in itertools.product(*cells):
        pts, wts = [], []
        for d, c in enumerate(cell):
            a, b = fine_nodes[d][c], fine_nodes[d][c + 1]
            pts.append(np.array([a, (a + b) / 2, b]))
            wts.append(simpson * (b - a))
        # values of all 1D hats at the 3 points, per axis
        lv = [np.array([_hat_eval(left_nodes[d], j, pts[d]) for j in range(lsz[d])]) for d in range(D)]
        rv = [np.array([_hat_eval(right_nodes[d], j, pts[d]) for j in range(rsz[d])]) for d in range(D)]
        for q in itertools.product(range(3), repeat=D):
            w = np.prod([wts[d][q[d]] for d in range(D)])
            lvals = np.ones(1)
            rvals = np.ones(1)
            for d in range(D):
                lvals = np.multiply.outer(lvals, lv[d][:, q[d]]).reshape(-1)
                rvals = np.multiply.outer(rvals, rv[d][:, q[d]]).reshape(-1)
            G += w * np.outer(lvals, rvals)
    return G


def _dense_projection(fine_nodes, coarse_nodes, u_fine):
    Gcc = _gram(fine_nodes, coarse_nodes, coarse_nodes)
    Gcf = _gram(fine_nodes, coarse_nodes, fine_nodes)
    return np.linalg.solve(Gcc, Gcf @ u_fine.reshape(-1))


@pytest.mark.parametrize("shape", [(5,), (9,), (6,), (5, 6), (5, 5, 9), (3, 3, 3, 3)])
def test_corrected_coarse_values_equal_dense_projection(shape):
    h = grid.hierarchy(shape, max_levels=1)
    u = np.random.default_rng(3).standard_normal(shape)
    v = multilevel.decompose(u, max_levels=1)
    fine = [h.coords(1, d) for d in range(h.D)]
    coarse = [h.coords(0, d) for d in range(h.D)]
    proj = _dense_projection(fine, coarse, u)
    got = v[np.ix_(*h.idx[0])].reshape(-1)
    assert np.max(np.abs(got - proj)) < 1e-12


@pytest.mark.parametrize("shape", [(9,), (17,), (9, 9), (9, 6, 5)])
def test_level0_values_equal_direct_projection(shape):
    """After the full recursion the level-0 values equal the projection of u
    straight onto V_0 (Q_0 Q_1 ... Q_L = Q_0 for nested spaces)."""
    h = grid.hierarchy(shape)
    u = np.random.default_rng(4).standard_normal(shape)
    v = multilevel.decompose(u)
    fine = [h.coords(h.L, d) for d in range(h.D)]
    coarse = [h.coords(0, d) for d in range(h.D)]
    proj = _dense_projection(fine, coarse, u)
    got = v[np.ix_(*h.idx[0])].reshape(-1)
    assert np.max(np.abs(got - proj)) < 1e-11


@pytest.mark.parametrize("shape", [(9,), (9, 6), (5, 5, 5)])
def test_level_norms_equal_quadrature(shape):
    """||Q_l u||^2 from the oracle's mass norm equals the quadrature of the
    square of the P1 function; orthogonal increments are nonnegative."""
    h = grid.hierarchy(shape)
    u = np.random.default_rng(5).standard_normal(shape)
    Q = multilevel.projections(u)
    fine = [h.coords(h.L, d) for d in range(h.D)]
    prev = 0.0
    for l in range(h.L + 1):
        nodes = [h.coords(l, d) for d in range(h.D)]
        G = _gram(fine, nodes, nodes)
        direct = float(Q[l].reshape(-1) @ G @ Q[l].reshape(-1))
        ours = multilevel.mass_norm2(h, l, Q[l])
        assert abs(direct - ours) < 1e-11 * max(1.0, abs(direct))
        assert ours >= prev - 1e-12
        prev = ours
