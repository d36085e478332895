"""GPU parity: every step of the CUDA path against the FP64 oracle, through
the C ABI (Python binding = argument marshalling only)."""
import math

import numpy as np
import pytest
import torch

from oracle import bounds, grid, huffman, multilevel, pipeline, quantize
from paper_2401_05994_b300 import binding, synth

from paper_2401_05994_b300.fmt import parse

pytestmark = pytest.mark.gpu

DEV = "cuda"

SHAPES = [(1000,), (9,), (129, 129), (33, 20), (47, 65, 33), (17, 17, 17), (9, 6, 5, 7),
          (1, 40, 1, 27), (7, 2), (1,), (3, 3, 3), (2000,), (5, 1100)]


def _field(shape, dtype, seed=0):
    if len(shape) >= 2 and min(shape) > 8:
        u = synth.gaussian_random_field(shape, beta=5.0 / 3.0, seed=seed, out_dtype=torch.float64)
    else:
        u = torch.from_numpy(np.random.default_rng(seed).standard_normal(shape))
    return u.to(dtype)


def _per_level_error(v_gpu, v_ref, shape):
    a = multilevel.level_coefficients(v_gpu)
    b = multilevel.level_coefficients(v_ref)
    return [(float(np.max(np.abs(x - y))) if x.size else 0.0,
             float(np.max(np.abs(y))) if y.size else 0.0) for x, y in zip(a, b)]


@pytest.mark.parametrize("shape", SHAPES)
def test_decompose_fp64_matches_oracle(shape):
    u = _field(shape, torch.float64, 1)
    ref = multilevel.decompose(u.numpy())
    got = binding.decompose(u.to(DEV).clone()).cpu().numpy()
    scale = max(1.0, float(np.max(np.abs(u.numpy()))))
    assert np.max(np.abs(got - ref)) <= 1e-11 * scale


@pytest.mark.parametrize("shape", SHAPES)
def test_decompose_fp32_per_level_tolerance(shape):
    u = _field(shape, torch.float32, 2)
    ref = multilevel.decompose(u.double().numpy())
    got = binding.decompose(u.to(DEV).clone()).cpu().double().numpy()
    umax = float(np.max(np.abs(u.numpy())))
    for err, cmax in _per_level_error(got, ref, shape):
        # 1e-5 of the level's largest coefficient, floored at a few float32
        # ulps of the data (a coefficient cannot be more accurate than u)
        assert err <= max(1e-5 * cmax, 8 * 2.0 ** -24 * umax)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape", SHAPES)
def test_recompose_inverts_and_matches_oracle(shape, dtype):
    rng = np.random.default_rng(3)
    v = rng.standard_normal(shape)
    ref = multilevel.recompose(v)
    got = binding.recompose(torch.from_numpy(v).to(dtype).to(DEV)).cpu().double().numpy()
    tol = 1e-11 if dtype == torch.float64 else 2e-5
    assert np.max(np.abs(got - ref)) <= tol * max(1.0, np.max(np.abs(ref)))
    u = _field(shape, dtype, 4).to(DEV)
    back = binding.recompose(binding.decompose(u.clone()))
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert float((back - u).abs().max()) <= tol * max(1.0, float(u.abs().max()))


@pytest.mark.parametrize("dtype,precision", [(torch.float32, "f32"), (torch.float64, "f64")])
@pytest.mark.parametrize("shape", [(129, 129), (47, 65, 33), (9, 6, 5, 7), (1000,)])
def test_quantize_bit_exact(shape, dtype, precision):
    u = _field(shape, dtype, 5)
    v = binding.decompose(u.to(DEV).clone())
    tau = 1e-3 * float(u.abs().max())
    w = binding.bin_widths(shape, tau, math.inf)
    sym, esc, hist = binding.quantize(v, w)
    rs, ro, rh = quantize.quantize(v.cpu().double().numpy() if precision == "f64"
                                   else v.cpu().numpy(), w, precision=precision)
    s_np = sym.cpu().numpy()
    assert np.array_equal(s_np, rs)
    assert np.array_equal(hist.cpu().numpy().astype(np.uint64), rh)
    esc_np = esc.cpu().numpy()
    assert np.array_equal(esc_np[s_np == 0], ro)
    # dequantize back into the in-place layout, bit-exact with the oracle
    back = binding.dequantize(sym, esc, shape, dtype, w).cpu().numpy()
    lv = quantize.dequantize_levels(rs, ro, quantize.level_counts(shape), w, precision)
    ref = quantize.scatter_levels(lv, shape)
    assert np.array_equal(back.astype(np.float64), ref)


def test_quantize_escapes_and_range():
    u = _field((65, 65), torch.float32, 6).to(DEV)
    v = binding.decompose(u.clone())
    w = binding.bin_widths(u.shape, 1e-7 * float(u.abs().max()), math.inf)
    sym, esc, hist = binding.quantize(v, w)
    s = sym.cpu().numpy()
    assert (s == 0).sum() > 0
    rs, ro, rh = quantize.quantize(v.cpu().numpy(), w, precision="f32")
    assert np.array_equal(s, rs) and np.array_equal(esc.cpu().numpy()[s == 0], ro)
    with pytest.raises(binding.MgardError) as e:
        binding.quantize(v, np.full_like(w, 1e-30))
    assert e.value.status == 11


def _hist_cases():
    rng = np.random.default_rng(7)
    out = []
    for k in range(6):
        h = np.zeros(4096, dtype=np.int64)
        n = int(rng.integers(2, 4096))
        sel = rng.choice(4096, n, replace=False)
        h[sel] = rng.geometric(0.001 if k % 2 else 0.3, n)
        out.append(h)
    fib = [1, 1]
    while len(fib) < 45:
        fib.append(fib[-1] + fib[-2])
    h = np.zeros(4096, dtype=np.int64)
    h[100:145] = fib
    out.append(h)                        # triggers the length limit
    h = np.zeros(4096, dtype=np.int64)
    h[2048] = 12345
    out.append(h)                        # single symbol
    h = np.zeros(4096, dtype=np.int64)
    h[[0, 7]] = [5, 5]
    out.append(h)
    out.append(np.ones(4096, dtype=np.int64))
    # many equal weights: ties between leaves and internal nodes everywhere
    h = np.zeros(4096, dtype=np.int64)
    sel = rng.choice(4096, 4000, replace=False)
    h[sel] = rng.integers(1, 4, 4000)
    out.append(h)
    h = np.zeros(4096, dtype=np.int64)
    sel = rng.choice(4096, 3000, replace=False)
    h[sel] = 2 ** rng.integers(0, 20, 3000)
    out.append(h)
    # total above 2^32 (64-bit merge weights)
    h = np.zeros(4096, dtype=np.int64)
    h[rng.choice(4096, 64, replace=False)] = rng.integers(2 ** 28, 2 ** 30, 64)
    out.append(h)
    # shaped like a quantized field: a sharp peak at the centre and a long tail of ones
    k = np.arange(4096)
    h = np.floor(1.0e8 * np.exp(-np.abs(k - 2048) / 6.0)).astype(np.int64)
    h[h == 0] = 1
    h[0] = 777
    out.append(h)
    return out


@pytest.mark.parametrize("case", range(14))
def test_codebook_matches_oracle(case):
    h = _hist_cases()[case]
    lengths, codes = binding.huffman_codebook(torch.from_numpy(h).to(DEV))
    ref = huffman.code_lengths(h)
    assert np.array_equal(lengths.cpu().numpy(), ref)
    rc = huffman.canonical_codes(ref).astype(np.uint32)
    got = codes.cpu().numpy().view(np.uint32)
    used = ref > 0
    assert np.array_equal(got[used], rc[used])


@pytest.mark.parametrize("n", [1, 1023, 1024, 1025, 70001, 9000])
def test_encode_decode_bit_exact(n):
    rng = np.random.default_rng(n)
    s = np.minimum(rng.geometric(0.05, n) + 2040, 4095).astype(np.uint16)
    s[rng.random(n) < 0.01] = 0
    if n == 9000:   # chunks of the zero symbol only (stored without words), incl. the last
        s[1024:3072] = 2048
        s[8192:] = 2048
    elif n == 70001:
        s[5 * 1024:6 * 1024] = 2048
    hist = np.bincount(s, minlength=4096)
    L = huffman.code_lengths(hist)
    esc = np.zeros(n, dtype=np.int32)
    esc[s == 0] = rng.integers(-10 ** 6, 10 ** 6, int((s == 0).sum()))
    st = torch.from_numpy(s.astype(np.int32)).to(torch.uint16).to(DEV)
    words, woff, eoff, sub, outl = binding.huffman_encode(st, torch.from_numpy(L).to(DEV),
                                                          torch.from_numpy(esc).to(DEV))
    rw, rwo, reo, rsub = huffman.encode(s, L, fill_symbol=2048)
    assert np.array_equal(words.cpu().numpy().view(np.uint32), rw)
    assert np.array_equal(woff.cpu().numpy().astype(np.uint64), rwo)
    assert np.array_equal(eoff.cpu().numpy().astype(np.uint64), reo)
    assert np.array_equal(sub.cpu().numpy().astype(np.uint16), rsub)
    assert np.array_equal(outl.cpu().numpy(), esc[s == 0])
    ds, de = binding.huffman_decode(words, woff, eoff, sub, torch.from_numpy(L).to(DEV), n, outl)
    d = ds.cpu().numpy()
    assert np.array_equal(d, s)
    assert np.array_equal(de.cpu().numpy()[d == 0], esc[s == 0])


@pytest.mark.parametrize("case", [5, 6, 11, 13])
def test_decode_long_codes_bit_exact(case):
    """Streams dominated by codes longer than the decoder's 14-bit prefix
    table, whose entries give the length when every code under a prefix has
    the same one and leave a search otherwise.  The codebooks: geometric
    weights (75 one-length prefixes, 4 mixed), the length-limited Fibonacci
    codes (up to 32 bits, one mixed prefix), the spread of 2^k weights (140
    and 7) and the quantized-field shape with its tail of ones, escape
    symbol included (6 and 2).  Symbols are drawn from the used ones, long
    codes favoured; the library's encoder must give the oracle's stream and
    its decoder must give back every symbol and escape value."""
    h = _hist_cases()[case]
    L = huffman.code_lengths(h)
    used = np.flatnonzero(L > 0)
    assert L.max() > 14
    rng = np.random.default_rng(case)
    w = 2.0 ** (L[used] - L[used].min())   # longer codes drawn more often
    n = 50001
    s = rng.choice(used, n, p=w / w.sum()).astype(np.uint16)
    esc = np.zeros(n, dtype=np.int32)
    if L[0] > 0:
        esc[s == 0] = rng.integers(-10 ** 6, 10 ** 6, int((s == 0).sum()))
    st = torch.from_numpy(s.astype(np.int32)).to(torch.uint16).to(DEV)
    Ld = torch.from_numpy(L).to(DEV)
    words, woff, eoff, sub, outl = binding.huffman_encode(st, Ld, torch.from_numpy(esc).to(DEV))
    rw, rwo, reo, rsub = huffman.encode(s, L, fill_symbol=2048)
    assert np.array_equal(words.cpu().numpy().view(np.uint32), rw)
    assert np.array_equal(woff.cpu().numpy().astype(np.uint64), rwo)
    ds, de = binding.huffman_decode(words, woff, eoff, sub, Ld, n, outl)
    assert np.array_equal(ds.cpu().numpy(), s)
    if L[0] > 0:
        d = ds.cpu().numpy()
        assert np.array_equal(de.cpu().numpy()[d == 0], esc[s == 0])


@pytest.mark.parametrize("s", [math.inf, 0.0, 1.0])
@pytest.mark.parametrize("case", ["c1_2d_f64", "grf_3d_f32", "uneven_3d_f32"])
def test_compress_round_trip_meets_bound(case, s):
    if case == "c1_2d_f64":
        u = torch.from_numpy(synth.sinusoids_2d(129, 129, seed=0))
    elif case == "grf_3d_f32":
        u = synth.gaussian_random_field((65, 65, 65), seed=1)
    else:
        u = synth.gaussian_random_field((37, 50, 29), beta=3.0, seed=2)
    tol = 1e-3
    ud = u.to(DEV)
    buf = binding.compress(ud, tol, s)
    meta = binding.info(buf)
    out = binding.decompress(buf)
    un = u.double().numpy()
    outn = out.cpu().double().numpy()
    # error measured in FP64 by the oracle's norm
    err = pipeline.error(un, outn, s)
    assert err <= meta["tol_abs"]
    ref_norm = bounds.norm(un, s)
    assert abs(meta["tol_abs"] - tol * ref_norm) <= 1e-5 * tol * ref_norm
    # device error norm agrees with the oracle's
    gerr = binding.error_norm(ud, out, s)
    assert abs(gerr - err) <= 1e-9 * max(err, 1e-30) + 1e-12
    # the payload equals the oracle encoder fed the GPU's symbols
    h, sec = parse(buf.cpu().numpy().tobytes())
    v = binding.decompose(ud.clone())
    sym, esc, hist = binding.quantize(v, sec["widths"])
    rl = huffman.code_lengths(hist.cpu().numpy())
    assert np.array_equal(sec["lengths"], rl)
    rw, rwo, reo, rsub = huffman.encode(sym.cpu().numpy(), rl, fill_symbol=2048)
    assert np.array_equal(sec["words"], rw)
    assert np.array_equal(sec["word_off"], rwo) and np.array_equal(sec["esc_off"], reo)
    assert np.array_equal(sec["sub_off"], rsub)
    sn = sym.cpu().numpy()
    assert np.array_equal(sec["outliers"], esc.cpu().numpy()[sn == 0])
    # widths equal the oracle's for the stored tolerance
    assert np.allclose(sec["widths"], bounds.bin_widths(u.shape, meta["tol_abs"], s), rtol=1e-12)


# Shapes of the pipeline parity test: the 129^3 cube, and three grids whose
# 513-node axis takes, in turn, the strided positions and the contiguous one
# (two-part restriction on 513-node strided lines, 257-node contiguous
# solves), as the 513^3 benchmark field does on its finest level.
PIPELINE_SHAPES = [(129, 129, 129), (513, 9, 40), (40, 513, 17), (9, 17, 513)]


def _integer_indices(sym, outliers):
    """Quantized integers q from symbols (q + 2048, or 0 for an escape whose
    value is the next outlier in symbol order)."""
    q = sym.astype(np.int64) - 2048
    esc = sym == 0
    q[esc] = outliers
    return q


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", PIPELINE_SHAPES)
def test_compressed_indices_match_fp64_oracle(shape, dtype, capsys):
    """The compress path the benchmark times (symbol-order coefficients,
    device buffers, second call replayed from the captured graph) against the
    FP64 oracle on the same input.

    * The stream decodes (library decoder) to symbols that the oracle's
      encoder turns back into the same words, offsets and outliers.
    * The decoded indices equal the oracle's FP64 quantization of its FP64
      coefficients.  FP64 data: at most 1e-6 of them may differ.  FP32 data:
      an index may differ only by one and only where the oracle's c/w lies
      within the float32 error of the coefficients of a half-integer; the
      count is reported and bounded by twice the expected number of such
      crossings (the summed per-node error in bins: a value whose c/w is off
      by d bins crosses a rounding boundary with probability d), plus a few.
    * Decompression equals the oracle's FP64 dequantization and
      recomposition of the same indices, to float32 rounding.
    """
    u = synth.gaussian_random_field(shape, seed=21, out_dtype=torch.float64).to(dtype)
    ud = u.to(DEV).contiguous()
    comp = torch.empty(binding.compress_bound(shape, dtype), dtype=torch.uint8, device=DEV)
    for _ in range(2):
        buf = binding.compress(ud, 1e-3, math.inf, binding.REL, out=comp)
    h, sec = parse(buf.cpu().numpy().tobytes())
    n = int(np.prod(shape))
    t = lambda a: torch.from_numpy(np.array(a)).to(DEV)
    sym_d, _ = binding.huffman_decode(t(sec["words"]), t(sec["word_off"]), t(sec["esc_off"]),
                                      t(sec["sub_off"]), t(sec["lengths"]), n, t(sec["outliers"]))
    sym = sym_d.cpu().numpy()
    rw, rwo, reo, rsub = huffman.encode(sym, sec["lengths"], fill_symbol=2048)
    assert np.array_equal(sec["words"], rw)
    assert np.array_equal(sec["word_off"], rwo) and np.array_equal(sec["esc_off"], reo)
    assert np.array_equal(sec["sub_off"], rsub)
    assert np.array_equal(sec["lengths"], huffman.code_lengths(np.bincount(sym, minlength=4096)))
    q_gpu = _integer_indices(sym, sec["outliers"])

    u64 = u.double().numpy()
    tol_abs = 1e-3 * float(np.max(np.abs(u64)))
    assert abs(h["tol_abs"] - tol_abs) <= 1e-15 * tol_abs
    w = bounds.bin_widths(shape, tol_abs, math.inf)
    assert np.allclose(sec["widths"], w, rtol=1e-12, atol=0)
    v64 = multilevel.decompose(u64)
    rs, ro, _ = quantize.quantize(v64, w, precision="f64")
    q_ref = _integer_indices(rs, ro)
    mism = np.nonzero(q_gpu != q_ref)[0]
    c64 = np.concatenate(multilevel.level_coefficients(v64))
    if dtype == torch.float64:
        assert len(mism) <= 1e-6 * n, len(mism)
    else:
        assert np.all(np.abs(q_gpu[mism] - q_ref[mism]) == 1)
        # per-node float32 error of the coefficients (the library's in-place
        # decomposition runs the same arithmetic as the symbol-order path)
        cg = np.concatenate(multilevel.level_coefficients(
            binding.decompose(ud.clone()).cpu().double().numpy()))
        wl = np.concatenate([np.full(k, w[l]) for l, k in
                             enumerate(quantize.level_counts(shape))])
        dx = np.abs(cg - c64) / wl
        x = c64[mism] / wl[mism]
        band = 2.0 * np.max(dx) + 1e-6
        assert np.all(np.abs(np.abs(x - np.floor(x)) - 0.5) <= band)
        expected = float(np.sum(np.minimum(dx, 0.5)))
        assert len(mism) <= 2.0 * expected + 5, (len(mism), expected)
        with capsys.disabled():
            print(f"\n[indices] {shape} f32: {len(mism)} of {n} differ from FP64 "
                  f"({len(mism) / n:.2e}; expected crossings {expected:.1f}; "
                  f"max coefficient error {np.max(dx):.2e} bins)")
    # decompression against the oracle's FP64 recomposition of the same indices
    out = binding.decompress(buf).cpu().double().numpy()
    lv = quantize.dequantize_levels(sym, sec["outliers"], quantize.level_counts(shape), w, "f64")
    ref = multilevel.recompose(quantize.scatter_levels(lv, shape))
    rtol = 1e-11 if dtype == torch.float64 else 2e-5
    assert np.max(np.abs(out - ref)) <= rtol * max(1.0, float(np.max(np.abs(ref))))
    assert np.max(np.abs(out - u64)) <= tol_abs


def test_host_buffers_round_trip():
    u = synth.gaussian_random_field((40, 33, 31), seed=9).numpy()
    buf = binding.compress(u, 1e-3)
    assert isinstance(buf, np.ndarray)
    out = binding.decompress(buf)
    assert isinstance(out, np.ndarray) and out.dtype == np.float32
    meta = binding.info(buf)
    assert np.max(np.abs(out.astype(np.float64) - u)) <= meta["tol_abs"]
    # device copy of the same buffer decompresses to the same values
    out_d = binding.decompress(torch.from_numpy(buf.copy()).to(DEV))
    assert np.array_equal(out_d.cpu().numpy(), out)


def test_nonfinite_and_bad_arguments():
    u = synth.gaussian_random_field((17, 17, 17), seed=3).to(DEV)
    u[3, 4, 5] = float("nan")
    with pytest.raises(binding.MgardError) as e:
        binding.compress(u, 1e-3)
    assert e.value.status == 4
    u[3, 4, 5] = 0.0
    with pytest.raises(binding.MgardError) as e:
        binding.compress(u, -1.0)
    assert e.value.status == 1
    with pytest.raises(binding.MgardError) as e:
        binding.compress(u, 1e-3, s=-2.0)
    assert e.value.status == 1


def test_corrupt_buffers_rejected():
    u = synth.gaussian_random_field((33, 33, 33), seed=4).to(DEV)
    buf = binding.compress(u, 1e-3).cpu().numpy()
    bad = buf.copy()
    bad[0] ^= 0xFF
    with pytest.raises(binding.MgardError) as e:
        binding.decompress(bad)
    assert e.value.status == 7
    with pytest.raises(binding.MgardError) as e:
        binding.decompress(buf[: len(buf) // 2].copy())
    assert e.value.status == 7
    h, sec = parse(buf.tobytes())
    # payload garbage: must either decode (it is only bits) or report corruption
    g = buf.copy()
    rng = np.random.default_rng(0)
    g[h["off_words"]:h["total_bytes"]] = rng.integers(0, 256, h["total_bytes"] - h["off_words"])
    try:
        binding.decompress(g)
    except binding.MgardError as e2:
        assert e2.status == 7
    # lengths that violate the Kraft inequality
    k = buf.copy()
    k[h["off_lengths"]:h["off_lengths"] + 4096] = 1
    with pytest.raises(binding.MgardError) as e:
        binding.decompress(k)
    assert e.value.status == 7
    # a sub-chunk start beyond its chunk
    so = buf.copy()
    so[h["off_sub_off"]:h["off_sub_off"] + 2] = 0xFF
    with pytest.raises(binding.MgardError) as e:
        binding.decompress(so)
    assert e.value.status == 7
    # chunk offsets past the payload
    o = buf.copy()
    o[h["off_word_off"] + 8:h["off_word_off"] + 16] = 0xFF
    with pytest.raises(binding.MgardError) as e:
        binding.decompress(o)
    assert e.value.status == 7


@pytest.mark.parametrize("s", [math.inf, 0.0, 1.0])
def test_norms_match_oracle(s):
    u = synth.gaussian_random_field((33, 40, 25), seed=5, out_dtype=torch.float64)
    got = binding.norm(u.to(DEV), s)
    ref = bounds.norm(u.numpy(), s)
    assert abs(got - ref) <= 1e-10 * ref


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape", [(220, 93, 244), (111, 47, 123)])
def test_shared_memory_limits_of_fused_kernels(shape, dtype):
    """Shapes whose fused restriction tiles need just under 48 KB of dynamic
    shared memory beside the kernel's static shared memory (a launch over
    the default limit fails); decomposition, recomposition and the s = 0
    norm (which decomposes in FP64) must all run and invert."""
    u = _field(shape, dtype, 6).to(DEV)
    v = binding.decompose(u.clone())
    back = binding.recompose(v)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert float((back - u).abs().max()) <= tol * max(1.0, float(u.abs().max()))
    e = binding.error_norm(u, back, 0.0)
    assert math.isfinite(e)


@pytest.mark.parametrize("shape", [(20001,), (3, 4001), (1100, 9, 5), (600, 3, 130)])
def test_fallback_paths_match_oracle(shape):
    """Shapes that leave the main kernels: lines of more than 1056 nodes
    (one thread per line), strided axes whose restriction tiles would not
    fit in shared memory (separate restriction and tile solve), and long
    thin grids.  FP64 decomposition against the oracle, FP32 per level,
    and a compress/decompress round trip within the bound."""
    u64 = _field(shape, torch.float64, 8)
    ref = multilevel.decompose(u64.numpy())
    got = binding.decompose(u64.to(DEV).clone()).cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-11 * max(1.0, float(np.max(np.abs(u64.numpy()))))
    u = u64.to(torch.float32)
    got32 = binding.decompose(u.to(DEV).clone()).cpu().double().numpy()
    umax = float(u.abs().max())
    for err, cmax in _per_level_error(got32, ref, shape):
        assert err <= max(1e-5 * cmax, 8 * 2.0 ** -24 * umax)
    ud = u.to(DEV)
    buf = binding.compress(ud, 1e-3, math.inf)
    out = binding.decompress(buf)
    err = pipeline.error(u.double().numpy(), out.cpu().double().numpy(), math.inf)
    assert err <= binding.info(buf)["tol_abs"]
