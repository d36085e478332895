"""Pins for the oracle's Huffman coder: Kraft equality, optimal cost against
an independent textbook (heap) construction, canonical-code properties,
the length limit, a hand-derived golden example and round trips."""
import heapq
import os

import numpy as np
import pytest

from oracle import huffman


def _textbook_cost(freq):
    """Total coded length of an optimal prefix code (heap-based Huffman)."""
    f = [int(x) for x in freq if x > 0]
    if len(f) == 1:
        return f[0]
    heapq.heapify(f)
    cost = 0
    while len(f) > 1:
        a = heapq.heappop(f)
        b = heapq.heappop(f)
        cost += a + b
        heapq.heappush(f, a + b)
    return cost


@pytest.mark.parametrize("seed", range(8))
def test_optimal_cost_and_kraft(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 4096))
    hist = np.zeros(4096, dtype=np.int64)
    sel = rng.choice(4096, n, replace=False)
    hist[sel] = rng.geometric(0.01, n) if seed % 2 else rng.integers(1, 5, n)
    L = huffman.code_lengths(hist).astype(np.int64)
    assert L.max() <= huffman.LMAX
    used = hist > 0
    assert np.all(L[used] > 0) and np.all(L[~used] == 0)
    kraft = sum(2.0 ** -int(x) for x in L[used])
    assert abs(kraft - 1.0) < 1e-12
    assert int((L * hist).sum()) == _textbook_cost(hist)


def test_canonical_codes_prefix_free_and_ordered():
    rng = np.random.default_rng(11)
    hist = rng.integers(0, 50, 300)
    L = huffman.code_lengths(hist).astype(int)
    C = huffman.canonical_codes(L).astype(int)
    syms = sorted(np.nonzero(L)[0], key=lambda s: (L[s], s))
    strs = [format(C[s], "0%db" % L[s]) for s in syms]
    for a in range(len(strs)):
        for b in range(len(strs)):
            if a != b:
                assert not strs[b].startswith(strs[a])
    for a, b in zip(syms, syms[1:]):
        if L[a] == L[b]:
            assert C[b] == C[a] + 1


def test_length_limit_triggers_and_holds():
    fib = [1, 1]
    while len(fib) < 45:
        fib.append(fib[-1] + fib[-2])
    hist = np.zeros(64, dtype=np.int64)
    hist[:45] = fib
    assert huffman._lengths_once(hist).max() > huffman.LMAX
    L = huffman.code_lengths(hist).astype(np.int64)
    assert L.max() <= huffman.LMAX
    assert abs(sum(2.0 ** -int(x) for x in L[L > 0]) - 1.0) < 1e-12


def test_single_symbol():
    hist = np.zeros(16, dtype=np.int64)
    hist[5] = 100
    L = huffman.code_lengths(hist)
    assert L[5] == 1 and L.sum() == 1
    words, off, esc, sub = huffman.encode(np.full(100, 5), L)
    assert len(words) == 4 and np.all(words == 0)


def test_golden_small_example():
    path = os.path.join(os.path.dirname(__file__), "golden", "huffman_small.txt")
    rec = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        rec[k] = v
    hist = np.zeros(64, dtype=np.int64)
    for kv in rec["hist"]:
        s, f = kv.split(":")
        hist[int(s)] = int(f)
    L = huffman.code_lengths(hist)
    C = huffman.canonical_codes(L)
    for kv in rec["lengths"]:
        s, v = kv.split(":")
        assert L[int(s)] == int(v)
    for kv in rec["codes"]:
        s, v = kv.split(":")
        assert C[int(s)] == int(v)
    words, off, _, _ = huffman.encode(np.array([int(t) for t in rec["stream"]]), L)
    assert [int(w) for w in words] == [int(x, 16) for x in rec["words"]]


@pytest.mark.parametrize("n", [0, 1, 1023, 1024, 1025, 5000])
def test_round_trip_with_chunks(n):
    rng = np.random.default_rng(n)
    sym = np.minimum(rng.geometric(0.2, n), 4095).astype(np.uint16)
    sym[::97] = 0
    hist = np.bincount(sym, minlength=4096)
    L = huffman.code_lengths(hist)
    words, off, esc, sub = huffman.encode(sym, L)
    assert len(off) == (n + 1023) // 1024
    if n:
        assert np.array_equal(huffman.decode(words, off, L, n), sym)
        # every sub-chunk decodes from its recorded start
        assert np.array_equal(huffman.decode(words, off, L, n, sub_off=sub), sym)
        for c in range(len(off)):
            seg = sym[c * 1024:(c + 1) * 1024]
            for k in range(1, 4):
                assert sub[c, 2 + k] == int(np.sum(seg[:k * 256] == 0))
        # escape prefix counts
        per_chunk = [int(np.sum(sym[c * 1024:(c + 1) * 1024] == 0)) for c in range(len(off))]
        assert esc.tolist() == list(np.concatenate([[0], np.cumsum(per_chunk)[:-1]]))


def test_fill_chunks_take_no_words():
    # chunk 0: only the fill symbol; chunk 1: mixed; chunk 2 (partial): only fill
    L = np.zeros(4096, dtype=np.int64)
    L[[2048, 2047, 2049]] = [1, 2, 2]
    sym = np.full(1024 * 2 + 300, 2048)
    sym[1024 + 5] = 2047
    sym[1024 + 900] = 2049
    words, off, esc, sub = huffman.encode(sym, L, fill_symbol=2048)
    # the mixed chunk alone: 1022 one-bit codes + two 2-bit codes = 1026 bits
    assert len(words) == (1026 + 31) // 32
    assert list(off) == [0, 0, len(words)]
    assert np.all(sub[0] == 0) and np.all(sub[2] == 0)
    assert np.array_equal(huffman.decode(words, off, L, len(sym), fill_symbol=2048), sym)
    assert np.array_equal(huffman.decode(words, off, L, len(sym), sub_off=sub, fill_symbol=2048), sym)
    # without the rule every chunk pays one bit per symbol
    w2, _, _, _ = huffman.encode(sym, L)
    assert len(w2) == 32 + (1026 + 31) // 32 + (300 + 31) // 32
