"""Compression pipeline assembled from the oracle's steps (test infrastructure).

Compression (paper, "Software design" and Listing 1): relative tolerances
are scaled by the norm of the data; the data is decomposed; every
coefficient is quantized with its level's bin width; the symbols are
Huffman-coded.  Decompression runs the steps backwards.  ``verify`` measures
the reconstruction error in FP64 in the norm the tolerance was given in.
"""
from __future__ import annotations

import math

import numpy as np

from . import bounds, huffman, multilevel, quantize
from .grid import hierarchy


def compress(u: np.ndarray, tol: float, s: float = math.inf, relative: bool = True,
             max_levels=None, precision: str = "f64"):
    u = np.asarray(u)
    h = hierarchy(u.shape, max_levels)
    tol_abs = tol * bounds.norm(u, s, max_levels) if relative else tol
    widths = bounds.bin_widths(u.shape, tol_abs, s, max_levels)
    v = multilevel.decompose(u, max_levels)
    symbols, outliers, hist = quantize.quantize(v, widths, max_levels, precision)
    lengths = huffman.code_lengths(hist)
    words, word_off, esc_off, sub_off = huffman.encode(symbols, lengths,
                                                        fill_symbol=quantize.R)
    return dict(shape=u.shape, L=h.L, tol_abs=tol_abs, widths=widths, s=s,
                symbols=symbols, outliers=outliers, hist=hist, lengths=lengths,
                words=words, word_off=word_off, esc_off=esc_off, sub_off=sub_off,
                precision=precision, max_levels=max_levels)


def decompress(c, symbols=None) -> np.ndarray:
    if symbols is None:
        symbols = huffman.decode(c["words"], c["word_off"], c["lengths"],
                                 len(c["symbols"]), fill_symbol=quantize.R)
    counts = quantize.level_counts(c["shape"], c["max_levels"])
    levels = quantize.dequantize_levels(symbols, c["outliers"], counts,
                                        c["widths"], c["precision"])
    v = quantize.scatter_levels(levels, c["shape"], c["max_levels"])
    return multilevel.recompose(v, c["max_levels"])


def compressed_bytes(c) -> int:
    """Size of the payload, code-length table, chunk offsets and outliers."""
    return (4 * len(c["words"]) + len(c["lengths"]) + 28 * len(c["word_off"])
            + 4 * len(c["outliers"]))


def error(u, u_hat, s: float = math.inf, max_levels=None) -> float:
    e = np.asarray(u_hat, dtype=np.float64) - np.asarray(u, dtype=np.float64)
    return bounds.norm(e, s, max_levels)
