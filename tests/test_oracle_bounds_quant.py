"""Pins for the oracle's error estimators and quantizer: operator norms
against brute-force operators, the bound on adversarial and random
quantization errors, rounding rules and the symbol layout."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import bounds, grid, multilevel, pipeline, quantize


def _correction_matrix_1d(n, l):
    """Dense matrix of the oracle's coarse correction on a 1D level, built by
    applying it to unit vectors (brute force)."""
    h = grid.hierarchy((n,))
    m = len(h.idx[l][0])
    cols = []
    for j in range(m):
        z = np.zeros(m)
        z[j] = 1.0
        cols.append(multilevel.correction(h, l, z))
    return np.array(cols).T, h


@pytest.mark.parametrize("n", [5, 6, 9, 17, 30])
def test_K_is_the_row_sum_norm_of_the_applied_correction(n):
    A, h = _correction_matrix_1d(n, grid.hierarchy((n,)).L)
    assert abs(np.abs(A).sum(axis=1).max() - bounds.K(h, h.L)) < 1e-12


@pytest.mark.parametrize("shape", [(9,), (9, 9), (9, 5, 6), (5, 5, 5, 5), (65, 65, 65)])
def test_K_below_classical_bound(shape):
    h = grid.hierarchy(shape)
    for l in range(1, h.L + 1):
        assert 0 < bounds.K(h, l) <= 3.0 ** h.D


def _level_error_maps(shape):
    """Per level l >= 1, the largest row sum of |R| over the columns of the
    level-l coefficients, R the exact map from coefficient errors to the
    reconstruction (every column a recomposition of a unit vector)."""
    h = grid.hierarchy(shape)
    lev = grid.node_level(h).reshape(-1)
    n = int(np.prod(shape))
    R = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        R[:, j] = multilevel.recompose(e.reshape(shape)).reshape(-1)
    A = np.abs(R)
    return h, [float(np.max(A[:, lev == l].sum(axis=1))) for l in range(1, h.L + 1)]


@pytest.mark.parametrize("shape,exact", [((65,), False), ((40,), False), ((33, 33), True),
                                         ((33, 20), False), ((9, 9, 9), True),
                                         ((9, 10, 11), True), ((5, 6, 7, 5), False)])
def test_linf_level_constant_against_brute_force(shape, exact):
    """c_l bounds every level's worst row of the exact error map; on these
    2D and 3D grids the class extremes meet at one row and c_l is that
    worst row itself."""
    h, brute = _level_error_maps(shape)
    for l, b in zip(range(1, h.L + 1), brute):
        c = bounds.linf_level_constant(h, l)
        assert b <= c * (1 + 1e-12), (l, b, c)
        if exact:
            assert abs(c - b) <= 1e-12 * c, (l, b, c)
        else:
            assert c <= 1.25 * b
        # never looser than the per-level bound 1 + K_l
        assert c <= 1.0 + bounds.K(h, l)


def _levels_and_masks(shape):
    h = grid.hierarchy(shape)
    lev = grid.node_level(h)
    return h, lev


@pytest.mark.parametrize("shape", [(17,), (9, 9), (9, 6, 5)])
def test_linf_bound_holds_for_adversarial_errors(shape):
    """Quantization errors of +-w/2 with the signs that maximise the error at
    one node: the error reaches a fair part of tau but never exceeds it."""
    h, lev = _levels_and_masks(shape)
    tau = 1.0
    w = bounds.bin_widths(shape, tau, math.inf)[0] / bounds.WIDTH_MARGIN
    n = int(np.prod(shape))
    # influence of each coefficient on every output node (recompose is linear)
    Rm = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Rm[:, j] = multilevel.recompose(e.reshape(shape)).reshape(-1)
    worst = np.abs(Rm).sum(axis=1).max() * w / 2
    assert worst <= tau * (1 + 1e-12)
    assert worst >= 0.1 * tau       # the bound is not vacuous
    i = int(np.argmax(np.abs(Rm).sum(axis=1)))
    delta = np.sign(Rm[i]) * w / 2
    err = np.abs(Rm @ delta).max()
    assert err <= tau * (1 + 1e-12)


@pytest.mark.parametrize("s", [math.inf, 0.0, 1.0])
@pytest.mark.parametrize("shape", [(33,), (17, 17), (9, 9, 9)])
def test_bound_holds_for_random_errors(shape, s):
    rng = np.random.default_rng(7)
    h, lev = _levels_and_masks(shape)
    tau = 0.3
    widths = bounds.bin_widths(shape, tau, s) / bounds.WIDTH_MARGIN
    for _ in range(5):
        delta = rng.uniform(-0.5, 0.5, size=shape) * widths[lev]
        e = multilevel.recompose(delta)
        assert bounds.norm(e, s) <= tau * (1 + 1e-12)


def test_s0_norm_is_l2_norm_of_p1_function():
    """For s = 0 the s-norm is the L2 norm of the interpolant; for a linear
    function on [0, 8] its square is the closed form integral."""
    x = np.arange(9, dtype=float)
    u = 2.0 * x - 3.0
    exact = ((2 * 8 - 3) ** 3 - (-3) ** 3) / (3 * 2.0)   # int_0^8 (2x-3)^2 dx
    assert abs(bounds.s_norm(u, 0.0) ** 2 - exact) < 1e-10



@pytest.mark.parametrize("shape", [(33,), (17, 9), (9, 10, 11)])
def test_s0_norm_telescopes_to_the_finest_energy(shape):
    """The level increments E_l - E_{l-1} are squared norms of differences of
    nested L2 projections, so none is negative and for s = 0 their sum is
    E_L = u^T M_L u: the norm needs the finest energy alone."""
    u = np.random.default_rng(len(shape)).standard_normal(shape).cumsum(axis=0)
    h = grid.hierarchy(shape)
    Q = bounds.projections(u)
    E = [bounds.mass_norm2(h, l, Q[l]) for l in range(h.L + 1)]
    assert all(E[l] >= E[l - 1] * (1 - 1e-12) for l in range(1, h.L + 1))
    EL = bounds.mass_norm2(h, h.L, u)
    assert abs(bounds.s_norm(u, 0.0) ** 2 - EL) <= 1e-12 * EL

def _snorm_golden():
    """Rows of tests/golden/snorm_1d.txt: hand-derived level energies of two
    fine-grid hats on x = 0..4 and the s-norm and width values built from
    them (derivations in the file)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "snorm_1d.txt")
    cases, widths = [], []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = [t.strip() for t in line.split("|")]
        if parts[0] == "widths":
            widths.append((float(parts[1]), float(parts[2]),
                           [float(Fraction(t)) for t in parts[3].split()]))
        else:
            cases.append((parts[0], np.array([float(t) for t in parts[1].split()]),
                          [float(Fraction(t)) for t in parts[2].split()],
                          [float(Fraction(t)) for t in parts[3].split()]))
    return cases, widths


def test_level_energies_match_hand_projections():
    """||Q_l u||^2 for l = 0, 1, 2 equals the values solved by hand from the
    normal equations of each level (pins the projections and the mass norm
    independently of the oracle's own operators)."""
    cases, _ = _snorm_golden()
    h = grid.hierarchy((5,))
    for _, u, E, _ in cases:
        Q = multilevel.projections(u)
        got = [multilevel.mass_norm2(h, l, Q[l]) for l in range(h.L + 1)]
        assert np.allclose(got, E, rtol=0, atol=1e-14), (got, E)


@pytest.mark.parametrize("k,s", [(0, 0.0), (1, 0.5), (2, 1.0)])
def test_s_norm_level_weighting_matches_golden(k, s):
    """The level weighting 4^{s l} with l = 0 the coarsest: the hand values
    separate it from 4^{s (L - l)} and 2^{s l}, and case B has all three
    level terms nonzero."""
    cases, _ = _snorm_golden()
    for name, u, _, S2 in cases:
        assert abs(bounds.s_norm(u, s) ** 2 - S2[k]) < 1e-13, (name, s)


@pytest.mark.parametrize("k,s", [(0, 0.0), (1, 0.5), (2, 1.0)])
def test_s_norm_of_separable_2d_field_is_product_of_1d_energies(k, s):
    """On the tensor-product grid 5 x 5 the projection of f(x) g(y) is
    Q_l f (x) Q_l g, so the level energies multiply: the 2D s-norm follows
    from the two 1D golden rows with no further derivation."""
    cases, _ = _snorm_golden()
    (_, fa, Ea, _), (_, fb, Eb, _) = cases
    u = np.outer(fa, fb)
    E = [a * b for a, b in zip(Ea, Eb)]
    exp = E[0] + sum(4.0 ** (s * l) * (E[l] - E[l - 1]) for l in (1, 2))
    assert abs(bounds.s_norm(u, s) ** 2 - exp) < 1e-13


def test_s_norm_bin_widths_match_golden():
    """w_l = 2 tau / sqrt((L+1) 4^{s l} mu_l n_l) with the Gershgorin bounds
    mu_l and new-node counts n_l worked out by hand for the shape (5,)."""
    _, widths = _snorm_golden()
    for s, tau, w2 in widths:
        w = bounds.bin_widths((5,), tau, s) / bounds.WIDTH_MARGIN
        assert np.allclose(w ** 2, w2, rtol=1e-14, atol=0), (s, w ** 2, w2)
    h = grid.hierarchy((5,))
    assert [bounds.mu(h, l) for l in range(3)] == [2.0, 2.0, 1.0]
    assert [h.new_count(l) for l in range(3)] == [2, 1, 2]


def test_rounding_ties_to_even_and_escapes():
    w = 0.5
    c = np.array([1.25, 0.75, -1.25, 2047.4 * w, 2047.6 * w, -3000 * w, 0.0])
    sym, out, hist = quantize.quantize_levels([c], [w])
    assert sym.tolist() == [2 + 2048, 2 + 2048, -2 + 2048, 2047 + 2048, 0, 0, 2048]
    assert out.tolist() == [2048, -3000]
    assert hist.sum() == len(c) and hist[0] == 2


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_dequantized_error_within_half_bound_width(precision):
    rng = np.random.default_rng(8)
    w = 3.7e-3
    c = rng.uniform(-9000 * w, 9000 * w, 40000)
    if precision == "f32":
        c = c.astype(np.float32)
    # points near half-integers are the hard cases, below and above the
    # float32-exact range of 4096 bins
    c[:2000] = ((rng.integers(-2047, 2047, 2000) + 0.5) * w).astype(c.dtype)
    c[2000:4000] = ((rng.integers(-4095, 4095, 2000) + 0.5) * w).astype(c.dtype)
    c[4000:4100] = ((rng.integers(4000, 4200, 100) + 0.5) * w).astype(c.dtype)
    sym, out, _ = quantize.quantize_levels([c], [w], precision)
    back = quantize.dequantize_levels(sym, out, [len(c)], [w], precision)[0]
    err = np.abs(back.astype(np.float64) - c.astype(np.float64))
    assert err.max() <= 0.5 * w / bounds.WIDTH_MARGIN


@pytest.mark.parametrize("shape", [(9, 6, 7), (17, 17), (5, 5, 5, 5)])
def test_symbol_layout_round_trip(shape):
    u = np.random.default_rng(9).standard_normal(shape)
    levels = multilevel.level_coefficients(u)
    assert [len(a) for a in levels] == quantize.level_counts(shape)
    assert sum(quantize.level_counts(shape)) == u.size
    back = quantize.scatter_levels(levels, shape)
    assert np.array_equal(back, u)


@pytest.mark.parametrize("s", [math.inf, 0.0, 1.0])
def test_pipeline_meets_tolerance(s):
    from paper_2401_05994_b300 import synth
    u = synth.sinusoids_2d(65, 65, seed=3)
    for tol in (1e-2, 1e-4):
        c = pipeline.compress(u, tol, s=s)
        ud = pipeline.decompress(c, symbols=c["symbols"])
        assert pipeline.error(u, ud, s) <= c["tol_abs"]
