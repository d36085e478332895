"""Huffman coding of quantization symbols (oracle; test infrastructure).

The paper ("Software design") ends the compression pipeline with lossless
encoding of the quantized coefficients into a self-describing buffer.  This
build uses a Huffman code.  Everything below is a specification choice,
since the paper fixes none of it:

Code lengths
    Leaves are the symbols of nonzero frequency, sorted by (frequency,
    symbol).  Two FIFO queues (leaves; internal nodes in creation order):
    repeatedly remove the two lightest heads (on equal weight the leaf queue
    goes first) and append their merged node to the internal queue.  A
    symbol's length is its leaf depth.  A single used symbol gets length 1.
    If the longest code exceeds ``LMAX = 32``, the construction is repeated
    on ``max(1, f >> k)`` for the smallest ``k >= 1`` that brings it within
    the limit.
Canonical codes
    Symbols sorted by (length, symbol) get consecutive code values; moving
    to a longer length shifts the running code left.
Stream layout
    Symbols are cut into chunks of ``CHUNK = 1024``.  Each chunk starts on a
    32-bit word boundary; code bits go MSB-first into each word.  Per chunk
    the stream records the exclusive prefix of word counts and of escape
    (outlier) counts, and, for its sub-chunks of ``SUB = 256`` symbols after
    the first, the bit offset inside the chunk where each starts and the
    number of escapes before it in the chunk (six uint16 per chunk), so the
    four sub-chunks of a chunk can be decoded independently.
Fill chunks
    With ``fill_symbol`` given (the compressor passes the symbol of q = 0),
    a chunk whose every symbol is ``fill_symbol`` is stored with no payload
    words and zero sub-chunk offsets; a decoder recognises it by its word
    count of 0 (any other nonempty chunk needs at least one word, since every
    code has at least one bit).  This keeps smooth regions from costing a bit
    per symbol.
"""
from __future__ import annotations

import numpy as np

LMAX = 32
CHUNK = 1024
SUB = 256


def _lengths_once(freq: np.ndarray) -> np.ndarray:
    used = np.nonzero(freq)[0]
    lengths = np.zeros(len(freq), dtype=np.int64)
    if len(used) == 0:
        return lengths
    if len(used) == 1:
        lengths[used[0]] = 1
        return lengths
    order = sorted(used.tolist(), key=lambda s: (int(freq[s]), s))
    n = len(order)
    leaf_w = [int(freq[s]) for s in order]
    # node ids: 0..n-1 leaves (sorted order), n.. internal nodes
    parent = [-1] * (2 * n - 1)
    int_w = []
    li, ii = 0, 0          # queue heads

    def take():
        nonlocal li, ii
        if li < n and (ii >= len(int_w) or leaf_w[li] <= int_w[ii]):
            li += 1
            return li - 1, leaf_w[li - 1]
        ii += 1
        return n + ii - 1, int_w[ii - 1]

    for k in range(n - 1):
        a, wa = take()
        b, wb = take()
        node = n + k
        parent[a] = node
        parent[b] = node
        int_w.append(wa + wb)
    depth = [0] * (2 * n - 1)
    for node in range(2 * n - 3, -1, -1):   # root (2n-2) has depth 0
        depth[node] = depth[parent[node]] + 1
    for i, s in enumerate(order):
        lengths[s] = depth[i]
    return lengths


def code_lengths(hist, lmax: int = LMAX) -> np.ndarray:
    freq = np.asarray(hist, dtype=np.int64)
    lengths = _lengths_once(freq)
    k = 0
    while lengths.max(initial=0) > lmax:
        k += 1
        f = np.where(freq > 0, np.maximum(1, freq >> k), 0)
        lengths = _lengths_once(f)
    return lengths.astype(np.uint8)


def canonical_codes(lengths) -> np.ndarray:
    lengths = np.asarray(lengths, dtype=np.int64)
    codes = np.zeros(len(lengths), dtype=np.uint64)
    syms = sorted(np.nonzero(lengths)[0].tolist(), key=lambda s: (lengths[s], s))
    code = 0
    prev = 0
    for i, s in enumerate(syms):
        ln = int(lengths[s])
        if i > 0:
            code += 1
        code <<= (ln - prev)
        prev = ln
        codes[s] = code
    return codes


def encode(symbols, lengths, esc_symbol: int = 0, chunk: int = CHUNK, fill_symbol=None):
    """Chunked MSB-first packing.

    Returns ``(words uint32, word_offsets uint64, esc_offsets uint64,
    sub_offsets uint16 [nchunks, 6])``; the offset arrays have one entry per
    chunk (exclusive prefixes)."""
    symbols = np.asarray(symbols, dtype=np.int64)
    lengths = np.asarray(lengths, dtype=np.int64)
    codes = canonical_codes(lengths).astype(np.uint64)
    n = len(symbols)
    nchunks = (n + chunk - 1) // chunk
    ln = lengths[symbols]
    if n and np.any(ln == 0):
        raise ValueError("symbol without a code")
    cid = np.arange(n) // chunk
    if fill_symbol is not None and n:
        not_fill = np.bincount(cid, weights=(symbols != fill_symbol), minlength=nchunks)
        fill_chunk = not_fill == 0
        ln = np.where(fill_chunk[cid], 0, ln)      # fill chunks emit no bits
    chunk_bits = np.bincount(cid, weights=ln, minlength=nchunks).astype(np.int64)
    chunk_words = (chunk_bits + 31) // 32
    word_off = np.zeros(nchunks, dtype=np.uint64)
    if nchunks:
        word_off[1:] = np.cumsum(chunk_words)[:-1]
    esc_cnt = np.bincount(cid, weights=(symbols == esc_symbol), minlength=nchunks).astype(np.int64)
    esc_off = np.zeros(nchunks, dtype=np.uint64)
    if nchunks:
        esc_off[1:] = np.cumsum(esc_cnt)[:-1]
    total = int(chunk_words.sum()) if nchunks else 0
    words = np.zeros(total + 1, dtype=np.uint64)   # one spare word for spill
    sub_off = np.zeros((nchunks, 6), dtype=np.uint16)
    if n:
        # offsets of the first symbol of sub-chunks 1..3 inside their chunk;
        # a sub-chunk past the end of the data starts at the chunk's end
        csum_bits = np.concatenate([[0], np.cumsum(ln)])
        csum_esc = np.concatenate([[0], np.cumsum(symbols == esc_symbol)])
        starts = np.arange(nchunks) * chunk
        for k in range(1, chunk // SUB):
            pos = np.minimum(starts + k * SUB, n)
            sub_off[:, k - 1] = csum_bits[pos] - csum_bits[starts]
            sub_off[:, 2 + k] = csum_esc[pos] - csum_esc[starts]
        # bit offset of each symbol inside its chunk
        csum = np.cumsum(ln)
        start_of_chunk = np.concatenate([[0], csum])[cid * chunk]
        bit_in_chunk = csum - ln - start_of_chunk
        gbit = word_off[cid].astype(np.int64) * 32 + bit_in_chunk
        emit = ln > 0
        w = gbit[emit] >> 5
        b = gbit[emit] & 31
        # place the code in a 64-bit window starting at word w (MSB first)
        sh = (64 - ln[emit] - b).astype(np.uint64)
        val = codes[symbols[emit]] << sh
        hi = val >> np.uint64(32)
        lo = val & np.uint64(0xFFFFFFFF)
        np.bitwise_or.at(words, w, hi)
        np.bitwise_or.at(words, w + 1, lo)
    return words[:total].astype(np.uint32), word_off, esc_off, sub_off


def decode(words, word_off, lengths, n: int, chunk: int = CHUNK, sub_off=None,
           fill_symbol=None) -> np.ndarray:
    """Bit-by-bit canonical decoding (slow; small inputs only).  With
    ``sub_off`` every sub-chunk starts from its recorded bit offset; with
    ``fill_symbol`` a chunk of zero words holds only that symbol."""
    lengths = np.asarray(lengths, dtype=np.int64)
    codes = canonical_codes(lengths)
    table = {(int(lengths[s]), int(codes[s])): s for s in np.nonzero(lengths)[0]}
    out = np.zeros(n, dtype=np.uint16)
    words = np.asarray(words, dtype=np.uint64)
    nchunks = (n + chunk - 1) // chunk
    for c in range(nchunks):
        nw = (int(word_off[c + 1]) if c + 1 < nchunks else len(words)) - int(word_off[c])
        if fill_symbol is not None and nw == 0:
            out[c * chunk:min(n, (c + 1) * chunk)] = fill_symbol
            continue
        for i in range(c * chunk, min(n, (c + 1) * chunk)):
            k = (i - c * chunk) // SUB
            if i == c * chunk or (sub_off is not None and (i - c * chunk) % SUB == 0):
                bit = int(word_off[c]) * 32 + (int(sub_off[c, k - 1]) if k else 0)
            code, ln = 0, 0
            while True:
                wv = int(words[bit >> 5])
                code = (code << 1) | ((wv >> (31 - (bit & 31))) & 1)
                bit += 1
                ln += 1
                if (ln, code) in table:
                    out[i] = table[(ln, code)]
                    break
                if ln > LMAX:
                    raise ValueError("corrupt stream")
    return out
