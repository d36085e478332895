"""Pins of the linear-QoI oracle: the integral functional's constant
representer and closed-form norm, the representer checked by exact Gauss
quadrature of the L2 inner product (independent of the mass matrices), the
duality bound with its equality case, and the QoI bound after compression."""
import math

import numpy as np
import pytest

from oracle import bounds, grid, multilevel, pipeline, qoi


def _trapezoid(shape):
    """Weights of the integral functional: the integral of each hat function,
    1/2 at the ends of an axis and 1 inside (unit spacing), tensor product."""
    w = np.ones(())
    for n in shape:
        a = np.ones(n)
        if n > 1:
            a[0] = a[-1] = 0.5
        w = np.multiply.outer(w, a)
    return w


@pytest.mark.parametrize("shape", [(9,), (17, 6), (9, 5, 7), (5, 1, 9)])
def test_integral_functional_has_constant_representer(shape):
    g = _trapezoid(shape)
    r = qoi.representer(g)
    assert np.max(np.abs(r - 1.0)) < 1e-12
    vol = float(np.prod([n - 1 for n in shape if n > 1]))
    # a constant lies in V_0: only the level-0 energy, the volume, remains
    for s in (0.0, 0.5, 1.0, 2.0):
        assert abs(qoi.norm(g, s) - math.sqrt(vol)) < 1e-10 * math.sqrt(vol)
    assert qoi.norm(g, math.inf) == vol


def _gauss_inner(shape, a, b):
    """Integral of the product of two P1 functions (nodal values a, b on the
    unit-spacing grid) by two-point Gauss quadrature on every cell, exact
    for products of multilinear functions."""
    t = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
    D = len(shape)
    total = 0.0
    for cell in np.ndindex(*[n - 1 for n in shape]):
        for q in np.ndindex(*([2] * D)):
            pt = [t[q[d]] for d in range(D)]
            va = vb = 0.0
            for corner in np.ndindex(*([2] * D)):
                wgt = 1.0
                for d in range(D):
                    wgt *= pt[d] if corner[d] else 1.0 - pt[d]
                idx = tuple(cell[d] + corner[d] for d in range(D))
                va += wgt * a[idx]
                vb += wgt * b[idx]
            total += va * vb / 2 ** D
    return total


@pytest.mark.parametrize("shape", [(7,), (6, 9), (3, 4, 5)])
def test_representer_reproduces_the_functional(shape):
    rng = np.random.default_rng(len(shape))
    g = rng.standard_normal(shape)
    r = qoi.representer(g)
    for _ in range(3):
        v = rng.standard_normal(shape)
        assert abs(_gauss_inner(shape, r, v) - qoi.value(v, g)) < 1e-10 * np.sum(np.abs(g))


def _components(r, max_levels=None):
    """Nodal values on the input grid of (Q_l - Q_{l-1}) r for every level."""
    h = grid.hierarchy(r.shape, max_levels)
    Q = multilevel.projections(r, max_levels)
    up = []
    for l in range(h.L + 1):
        U = Q[l]
        for k in range(l + 1, h.L + 1):
            U = multilevel.interpolate(h, k, U)
        up.append(U.reshape(r.shape))
    return [up[0]] + [up[l] - up[l - 1] for l in range(1, h.L + 1)]


@pytest.mark.parametrize("shape", [(33,), (17, 9), (9, 9, 5)])
@pytest.mark.parametrize("s", [0.0, 0.5, 1.0])
def test_duality_bound_and_its_equality_case(shape, s):
    rng = np.random.default_rng(7)
    g = rng.standard_normal(shape)
    nq = qoi.norm(g, s)
    for _ in range(4):
        e = rng.standard_normal(shape).cumsum(axis=0)
        assert abs(qoi.value(e, g)) <= nq * bounds.s_norm(e, s) * (1 + 1e-12)
    # equality for e = sum_l 4^{-s l} (Q_l - Q_{l-1}) r
    comps = _components(qoi.representer(g))
    e_star = sum(4.0 ** (-s * l) * c for l, c in enumerate(comps))
    lhs = qoi.value(e_star, g)
    assert abs(lhs - nq * bounds.s_norm(e_star, s)) <= 1e-9 * abs(lhs)
    # the dual norm of the L-infinity norm is the 1-norm of the weights
    e = np.sign(g)
    assert abs(qoi.value(e, g) - qoi.norm(g, math.inf) * np.max(np.abs(e))) < 1e-12 * np.sum(np.abs(g))


def _qois(shape, rng):
    box = np.zeros(shape)
    box[2:9, 3:8, 1:6] = 1.0 / (7 * 5 * 5)
    point = np.zeros(shape)
    point[8, 5, 4] = 1.0
    return {"box average": box, "random weights": rng.uniform(0.0, 1.0, shape) / np.prod(shape),
            "point value": point}


@pytest.mark.parametrize("s", [0.0, 1.0, math.inf])
def test_qoi_error_within_tolerance_after_compression(s):
    rng = np.random.default_rng(11)
    shape = (17, 12, 9)
    u = rng.standard_normal(shape).cumsum(axis=0).cumsum(axis=1)
    for name, g in _qois(shape, rng).items():
        for rel in (1e-2, 1e-4):
            tol = rel * float(np.max(np.abs(u)))
            c = qoi.compress(u, g, tol, s)
            assert c["tol_abs"] == tol / qoi.norm(g, s)
            err = abs(qoi.value(pipeline.decompress(c), g) - qoi.value(u, g))
            assert err <= tol, (name, rel, err / tol)
