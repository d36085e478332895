"""Pins of the refactoring oracle: a hand-worked bit-plane golden, the
truncation bound of every plane count, the L-infinity estimate against the
brute-force error of reconstructions (the error of recomposing truncated
coefficients never exceeds it), the greedy rule, and exact recovery with
every plane."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import mdr, multilevel


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "mdr_planes.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        parts = [p.split() for p in line.split("|")]
        c = np.array([float(Fraction(t)) for t in parts[0]])
        return (c, int(parts[1][0]), int(parts[2][0]), [int(t) for t in parts[3]],
                {1: [float(t) for t in parts[4]], 2: [float(t) for t in parts[5]],
                 4: [float(t) for t in parts[6]]})


def test_planes_and_reconstruction_match_hand_worked_level():
    c, e, sign_word, plane_words, rec = _golden()
    e2, signs, planes = mdr.encode_level(c, 4)
    assert e2 == e
    assert signs.tolist() == [sign_word]
    assert [int(p[0]) for p in planes] == plane_words
    for P, exp in rec.items():
        got = mdr.decode_level(len(c), e, signs, planes, P, 4)
        assert got.tolist() == exp, (P, got)


@pytest.mark.parametrize("B", [8, 20, 32])
def test_truncation_stays_within_the_level_bound(B):
    rng = np.random.default_rng(B)
    c = rng.standard_normal(1000) * np.exp(rng.uniform(-8, 3, 1000))
    c[::7] = 0.0
    e, signs, planes = mdr.encode_level(c, B)
    assert np.max(np.abs(c)) < 2.0 ** e <= 2 * np.max(np.abs(c))
    prev = math.inf
    for P in range(B + 1):
        d = np.max(np.abs(mdr.decode_level(len(c), e, signs, planes, P, B) - c))
        assert d < 2.0 ** (e - P)
        assert d <= prev * (1 + 1e-15) or P > 0 and d < 2.0 ** (e - P)
        prev = d
    # zeros stay zero once any plane is read, signs survive
    back = mdr.decode_level(len(c), e, signs, planes, B, B)
    assert np.all(back[::7] == 0.0)
    assert np.all(np.sign(back[np.abs(back) > 0]) == np.sign(c[np.abs(back) > 0]))


@pytest.mark.parametrize("shape", [(65,), (17, 33), (9, 10, 11)])
def test_estimate_bounds_the_reconstruction_error(shape):
    """Brute force: for plane selections along the greedy path and random
    ones, the FP64 error of the reconstruction never exceeds the estimate."""
    rng = np.random.default_rng(len(shape))
    u = rng.standard_normal(shape).cumsum(axis=-1)
    r = mdr.refactor(u, B=32)
    nl = len(r["counts"])
    for tol in (1.0, 1e-1, 1e-3, 1e-5, 1e-7):
        P, nbytes, est = mdr.request(r, tol)
        err = float(np.max(np.abs(mdr.reconstruct(r, P) - u)))
        assert est <= tol and err <= est
        assert nbytes == sum(4 * ((n + 31) // 32) * (1 + p) for n, p in zip(r["counts"], P) if p)
    for _ in range(5):
        P = [int(p) for p in rng.integers(0, 33, nl)]
        err = float(np.max(np.abs(mdr.reconstruct(r, P) - u)))
        assert err <= mdr.estimate(r, P)


def test_greedy_takes_the_largest_reduction_per_byte():
    u = np.random.default_rng(3).standard_normal((33, 17)).cumsum(axis=0)
    r = mdr.refactor(u, B=16)
    words = [(n + 31) // 32 for n in r["counts"]]
    P_prev = [0] * len(words)
    floor = mdr.estimate(r, [r["B"]] * len(words))   # every plane read
    for tol in np.geomspace(mdr.estimate(r, P_prev) * 0.99, 2 * floor, 25):
        P, _, est = mdr.request(r, tol)
        assert est <= tol
        # every level added relative to a looser request had a rate at least
        # that of any level not yet fully read at that point (checked on the
        # last plane of each level: its rate is the smallest it contributed)
        for l in range(len(P)):
            if P[l] == 0:
                continue
            rate_l = r["weights"][l] * 2.0 ** (r["exponents"][l] - P[l]) / (4 * words[l] * (2 if P[l] == 1 else 1))
            for k in range(len(P)):
                if k == l or P[k] >= r["B"] or not r["nonzero"][k]:
                    continue
                nxt = r["weights"][k] * 2.0 ** (r["exponents"][k] - P[k] - 1) / (4 * words[k] * (2 if P[k] == 0 else 1))
                assert rate_l >= nxt * (1 - 1e-12)
        P_prev = P


def test_every_plane_recovers_the_decomposition():
    u = np.random.default_rng(5).standard_normal((17, 9, 5))
    r = mdr.refactor(u, B=32)
    full = mdr.reconstruct(r, [32] * len(r["counts"]))
    est = mdr.estimate(r, [32] * len(r["counts"]))
    assert np.max(np.abs(full - u)) <= est
    assert est < 1e-8 * np.max(np.abs(u))
    # no planes: every coefficient reads as zero
    assert np.all(mdr.reconstruct(r, [0] * len(r["counts"])) == 0.0)
    # weights are the compressor's L-infinity weights
    v = multilevel.decompose(u)
    assert len(multilevel.level_coefficients(v)) == len(r["weights"])
    assert r["weights"][0] == 1.0 and all(w > 0.0 for w in r["weights"][1:])
