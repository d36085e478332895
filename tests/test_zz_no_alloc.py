"""The allocation-free Huffman encoder against the regular one.

`mgard_huffman_encode_noalloc` exists for callers that cannot allocate device
memory (for example code running under another framework's memory manager, or
where cudaMalloc is not permitted).  It keeps its scratch in a fixed device
array inside the library instead.  These checks call both entry points
through the C ABI on the same inputs and require identical streams, twice in a
row (the second call must not see stale scratch from the first), and check
with the library's allocation counter that those calls allocated nothing.  The
file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import huffman
from paper_2401_05994_b300 import binding

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    s = np.minimum(rng.geometric(0.02 + 0.03 * (seed % 3), n) + 2000, 4095).astype(np.uint16)
    s[rng.random(n) < 0.03] = 0
    esc = np.zeros(n, dtype=np.int32)
    esc[s == 0] = rng.integers(-(10 ** 7), 10 ** 7, int((s == 0).sum()))
    L = huffman.code_lengths(np.bincount(s, minlength=4096))
    return (torch.from_numpy(s.astype(np.int32)).to(torch.uint16).to(DEV),
            torch.from_numpy(L).to(DEV), torch.from_numpy(esc).to(DEV))


def _encode(fn, sym, lengths, esc):
    n = sym.numel()
    nchunks = (n + 1023) // 1024
    cap = n + nchunks + 1
    words = torch.full((cap,), -1, dtype=torch.int32, device=DEV)
    woff = torch.full((nchunks,), -1, dtype=torch.int64, device=DEV)
    eoff = torch.full((nchunks,), -1, dtype=torch.int64, device=DEV)
    sub = torch.zeros((nchunks, 6), dtype=torch.uint16, device=DEV)
    outl = torch.full((n,), -1, dtype=torch.int32, device=DEV)
    nw, no = ctypes.c_uint64(), ctypes.c_uint64()
    st = fn(ctypes.c_void_p(sym.data_ptr()), n, ctypes.c_void_p(lengths.data_ptr()),
            ctypes.c_void_p(esc.data_ptr()), ctypes.c_void_p(words.data_ptr()), cap,
            ctypes.c_void_p(woff.data_ptr()), ctypes.c_void_p(eoff.data_ptr()),
            ctypes.c_void_p(sub.data_ptr()), ctypes.c_void_p(outl.data_ptr()), n,
            ctypes.byref(nw), ctypes.byref(no),
            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, binding.lib().mgard_last_error()
    torch.cuda.synchronize()
    return (words[:nw.value].cpu().numpy(), woff.cpu().numpy(), eoff.cpu().numpy(),
            outl[:no.value].cpu().numpy(), nw.value, no.value, sub.cpu().numpy())


def test_noalloc_encode_matches_regular_encode_twice():
    L = binding.lib()
    L.mgard_device_allocations.restype = ctypes.c_uint64
    # a large call first, then a smaller one with a different code table
    cases = [_inputs(n, seed) for n, seed in ((3_000_001, 1), (70_001, 2))]
    refs = [_encode(L.mgard_huffman_encode, *c) for c in cases]
    # the library makes no allocation of any kind during the two calls
    allocs = L.mgard_device_allocations()
    gots = [_encode(L.mgard_huffman_encode_noalloc, *c) for c in cases]
    assert L.mgard_device_allocations() == allocs
    for (sym, lengths, esc), ref, got in zip(cases, refs, gots):
        n = sym.numel()
        assert ref[4] == got[4] and ref[5] == got[5]
        for a, b in zip(ref[:4] + ref[6:], got[:4] + got[6:]):
            assert np.array_equal(a, b)
        # and the stream decodes back to the symbols
        words = torch.from_numpy(got[0]).to(DEV)
        ds, _ = binding.huffman_decode(words, torch.from_numpy(got[1]).to(DEV),
                                       torch.from_numpy(got[2]).to(DEV),
                                       torch.from_numpy(got[6].astype(np.int32)).to(torch.uint16).to(DEV),
                                       lengths, n, torch.from_numpy(got[3]).to(DEV))
        assert torch.equal(ds.to(torch.int32), sym.to(torch.int32))


def test_noalloc_encode_rejects_oversized_input():
    """Sizes beyond the fixed scratch are refused before any device work."""
    L = binding.lib()
    buf = torch.zeros(16, dtype=torch.int32, device=DEV)
    p = ctypes.c_void_p(buf.data_ptr())
    nw, no = ctypes.c_uint64(), ctypes.c_uint64()
    too_many = 2048 * 4096 * 1024 + 1
    st = L.mgard_huffman_encode_noalloc(p, too_many, p, p, p, 0, p, p, p, p, 0, ctypes.byref(nw),
                                        ctypes.byref(no), None)
    assert st == 1
    assert b"mgard_huffman_encode" in L.mgard_last_error()
