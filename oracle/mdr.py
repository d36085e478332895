"""Multilevel data refactoring (oracle; test infrastructure).

The paper's "Software design" section describes a second pipeline beside
compression: the multilevel coefficients u_mc are refactored into precision
segments (bit-planes), an error estimate is accumulated per segment, and
retrieval picks segments greedily until the requested error is met; its
"APIs" section names the calls MDRefactor / MDRequest / MDReconstruct.  The
paper gives no formulas; this module writes out the reading used here, in
FP64, plainly:

Refactor (per level l, coefficients c in level order)
    ``e_l``  the smallest integer with max|c| < 2^e_l (``math.frexp``); a
             level whose coefficients are all zero has e_l = 0 and no error.
    ``q``    floor(|c| * 2^(B - e_l)), an integer below 2^B (B planes).
    plane b (b = 0 the most significant) holds bit B-1-b of every q; the
    sign plane holds c < 0.  Bits are packed 32 to a word, coefficient
    32 w + i in bit i of word w.

Reconstruct with P planes of level l
    q_P = q with its B-P low bits cleared; the value is 0 when q_P = 0, else
    (q_P + 2^(B-P-1)) 2^(e_l-B) (the middle of the truncation interval; with
    P = B, q_P 2^(e_l-B)), with the sign.  Every coefficient is then within
    2^(e_l-P) of c (strictly).

Error estimate (L-infinity)
    The recomposition bound of the compressor (see bounds.py): an error of
    at most d_l in the level-l coefficients gives at most
    ``sum_l w_l d_l`` with w_0 = 1 and w_l = c_l (the per-level constant of
    the L-infinity width).  With d_l = 2^(e_l-P_l)
    (0 for an all-zero level) that is the estimate of a plane selection.

Request (greedy)
    Start from no planes; while the estimate exceeds the tolerance, add the
    next plane of the level whose added plane lowers the estimate most per
    byte (a plane of level l costs ceil(n_l / 32) words, the first one also
    the sign plane's), ties to the lower level.
"""
from __future__ import annotations

import math

import numpy as np

from . import bounds, multilevel, quantize
from .grid import hierarchy


def exponent(c: np.ndarray) -> int:
    m = float(np.max(np.abs(c))) if c.size else 0.0
    if m == 0.0:
        return 0
    return math.frexp(m)[1]


def integers(c: np.ndarray, e: int, B: int) -> np.ndarray:
    """q = floor(|c| 2^(B - e)) as uint64 (exact: a power-of-two scaling)."""
    a = np.abs(np.asarray(c, dtype=np.float64))
    return np.floor(np.ldexp(a, B - e)).astype(np.uint64)


def pack(bits: np.ndarray) -> np.ndarray:
    """Bits (0/1 per coefficient) into uint32 words, bit i of word w for
    coefficient 32 w + i."""
    n = len(bits)
    nw = (n + 31) // 32
    padded = np.zeros(nw * 32, dtype=np.uint64)
    padded[:n] = bits
    sh = np.arange(32, dtype=np.uint64)
    return (padded.reshape(nw, 32) << sh).sum(axis=1).astype(np.uint32)


def unpack(words: np.ndarray, n: int) -> np.ndarray:
    w = np.asarray(words, dtype=np.uint64)
    sh = np.arange(32, dtype=np.uint64)
    return ((w[:, None] >> sh) & np.uint64(1)).reshape(-1)[:n]


def encode_level(c: np.ndarray, B: int):
    """(exponent, sign words, [plane words for b = 0..B-1])."""
    c = np.asarray(c, dtype=np.float64)
    e = exponent(c)
    q = integers(c, e, B)
    signs = pack((c < 0).astype(np.uint64))
    planes = [pack((q >> np.uint64(B - 1 - b)) & np.uint64(1)) for b in range(B)]
    return e, signs, planes


def decode_level(n: int, e: int, signs, planes, P: int, B: int) -> np.ndarray:
    """Coefficients from the first P planes (FP64)."""
    q = np.zeros(n, dtype=np.uint64)
    for b in range(P):
        q |= unpack(planes[b], n) << np.uint64(B - 1 - b)
    val = q.astype(np.float64)
    if P < B:
        half = float(2 ** (B - P - 1))
        val = np.where(q > 0, val + half, 0.0)
    val = np.ldexp(val, e - B)
    neg = unpack(signs, n).astype(bool)
    return np.where(neg, -val, val)


def weights(shape, max_levels=None) -> np.ndarray:
    """w_0 = 1, w_l = c_l (the L-infinity recomposition weights)."""
    h = hierarchy(shape, max_levels)
    return np.array([1.0] + [bounds.linf_level_constant(h, l) for l in range(1, h.L + 1)])


def refactor(u: np.ndarray, B: int = 32, max_levels=None):
    """Decompose u and bit-plane encode every level."""
    v = multilevel.decompose(u, max_levels)
    levels = multilevel.level_coefficients(v, max_levels)
    enc = [encode_level(c, B) for c in levels]
    return dict(shape=u.shape, B=B, max_levels=max_levels,
                counts=[len(c) for c in levels],
                exponents=[x[0] for x in enc], signs=[x[1] for x in enc],
                planes=[x[2] for x in enc], nonzero=[bool(np.any(c != 0)) for c in levels],
                weights=weights(u.shape, max_levels))


def level_bound(e: int, P: int, nonzero: bool) -> float:
    return math.ldexp(1.0, int(e) - int(P)) if nonzero else 0.0


def estimate(r, P) -> float:
    """sum_l w_l d_l, added left to right in level order (each term is exact:
    a power of two times w_l)."""
    total = 0.0
    for w, e, p, nz in zip(r["weights"], r["exponents"], P, r["nonzero"]):
        total += float(w) * level_bound(e, p, nz)
    return total


def request(r, tol: float):
    """Greedy plane counts per level, their bytes and the estimate."""
    B = r["B"]
    nl = len(r["counts"])
    P = [0] * nl
    words = [(n + 31) // 32 for n in r["counts"]]
    est = estimate(r, P)
    while est > tol:
        best, best_rate = -1, -1.0
        for l in range(nl):
            if P[l] >= B or not r["nonzero"][l]:
                continue
            gain = r["weights"][l] * (level_bound(r["exponents"][l], P[l], True) -
                                      level_bound(r["exponents"][l], P[l] + 1, True))
            cost = 4 * words[l] * (2 if P[l] == 0 else 1)
            rate = gain / cost
            if rate > best_rate:
                best, best_rate = l, rate
        if best < 0:
            break
        P[best] += 1
        est = estimate(r, P)
    nbytes = sum(4 * words[l] * (1 + P[l]) for l in range(nl) if P[l] > 0)
    return P, nbytes, est


def reconstruct(r, P) -> np.ndarray:
    """Decode P[l] planes of every level and recompose (FP64)."""
    levels = [decode_level(n, e, s, pl, p, r["B"])
              for n, e, s, pl, p in zip(r["counts"], r["exponents"], r["signs"], r["planes"], P)]
    v = quantize.scatter_levels(levels, r["shape"], r["max_levels"])
    return multilevel.recompose(v, r["max_levels"])
