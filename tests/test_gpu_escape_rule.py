"""Escapes of 4096 bins or more follow double-precision rules: the bin index
q = rint(fl64(c / w)) and the value fl32(fl64(q * w)).  The float kernels
take these decisions in two-float arithmetic and fall back to double only
where that arithmetic cannot prove the rounding; these tests compare them
with the rules evaluated by numpy in FP64, on inputs packed next to the
rounding boundaries (exact ties, near-ties on both sides), on random ones,
and on values outside the two-float range (huge q, widths beyond 2^+-60).
"""
import numpy as np
import pytest
import torch

from paper_2401_05994_b300 import binding

pytestmark = pytest.mark.gpu
DEV = "cuda"
ESC = 0


def _quantize(c, w):
    sym, esc, _ = binding.quantize(torch.from_numpy(c).to(DEV), [w], max_levels=0)
    return sym.cpu().numpy().astype(np.int64), esc.cpu().numpy()


def _dequantize(q, w):
    n = q.size
    sym = torch.full((n,), ESC, dtype=torch.uint16, device=DEV)
    esc = torch.from_numpy(q.astype(np.int32)).to(DEV)
    out = binding.dequantize(sym, esc, (n,), torch.float32, [w], max_levels=0)
    return out.cpu().numpy()


def _near(x, k):
    """x and its k float32 neighbours on each side."""
    vals = [x]
    up = dn = x
    for _ in range(k):
        up = np.nextafter(up, np.float32(np.inf))
        dn = np.nextafter(dn, np.float32(-np.inf))
        vals += [up, dn]
    return np.array(vals, dtype=np.float32)


def _quantize_cases(rng, w):
    """Coefficients c with |c / w| >= 4200 (decided by the double rule)."""
    cases = []
    # half-integers k + 1/2 times w, as floats, with neighbours on both sides
    for k in rng.integers(4200, 1 << 21, 400):
        c = np.float32(((int(k) + 0.5) * w))
        cases.append(_near(c, 3))
    # exact ties where w is a power of two: c / w = k + 1/2 exactly
    e = np.floor(np.log2(w))
    if w == 2.0 ** e:
        ks = rng.integers(4200, 1 << 20, 200)
        cases.append(((ks + 0.5) * w).astype(np.float32))
    # random magnitudes over the whole range, both signs
    r = rng.uniform(4200.0, 2.0 ** 21, 4000) * w
    cases.append(r.astype(np.float32))
    c = np.concatenate(cases)
    c = np.concatenate([c, -c])
    return c[np.abs(c.astype(np.float64) / w) >= 4200]


@pytest.mark.parametrize("w", [1.0, 2.0 ** -10, 0.1, 3.7e-3, 1e-7, 123.456, 2.0 ** -70, 2.0 ** 70])
def test_quantize_big_escapes_follow_double_rule(w):
    rng = np.random.default_rng(int(abs(np.log2(w)) * 1000) % 2 ** 31)
    c = _quantize_cases(rng, w)
    sym, esc = _quantize(c, w)
    ref = np.rint(c.astype(np.float64) / w)
    assert np.all(sym == ESC)
    ok = np.abs(ref) <= 2 ** 31 - 1
    assert np.array_equal(esc[ok].astype(np.int64), ref[ok].astype(np.int64))


def test_quantize_out_of_range_flags():
    c = np.array([5000.0, 3e12], dtype=np.float32)
    with pytest.raises(binding.MgardError):
        _quantize(c, 1.0)


def _dequantize_cases(rng, w):
    q = []
    # products next to float midpoints: w chosen so that q * w lands there
    # is done per width below; here random and extreme indices
    q.append(rng.integers(4096, 1 << 24, 4000))
    q.append(rng.integers(1 << 24, 2 ** 31 - 1, 200))
    q.append(np.array([4096, 4097, (1 << 24) - 1, 1 << 24, (1 << 24) + 1, 2 ** 31 - 1]))
    q = np.concatenate(q)
    return np.concatenate([q, -q])


@pytest.mark.parametrize("w", [1.0, 0.1, 3.7e-3, 1e-7, 123.456, 2.0 ** -70, 2.0 ** 70])
def test_dequantize_big_escapes_follow_double_rule(w):
    rng = np.random.default_rng(7)
    q = _dequantize_cases(rng, w)
    got = _dequantize(q, w)
    ref = (q.astype(np.float64) * w).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_dequantize_products_at_float_midpoints():
    """Per q, a width that puts q * w on a float midpoint in double, or one
    double ulp to either side: the double rounding decides these."""
    rng = np.random.default_rng(11)
    q = rng.integers(4096, 1 << 24, 120)
    f = (rng.uniform(1.0, 2.0, q.size) * 2.0 ** 10).astype(np.float32)
    mids = f.astype(np.float64) + np.spacing(f).astype(np.float64) / 2
    for qq, mm in zip(q, mids):
        w0 = float(mm / qq)
        for w in (float(np.nextafter(w0, -np.inf)), w0, float(np.nextafter(w0, np.inf))):
            a = np.array([qq, -qq])
            got = _dequantize(a, w)
            ref = (a.astype(np.float64) * w).astype(np.float32)
            assert np.array_equal(got.view(np.uint32), ref.view(np.uint32)), (qq, w)


@pytest.mark.parametrize("w", [3 * 2.0 ** -22, 5 * 2.0 ** -23, 7 * 2.0 ** -21, 2.0 ** -20])
def test_dequantize_exact_products(w):
    """Widths with few significant bits make q * w exact in double, and a
    share of them exact float midpoints (ties to even)."""
    rng = np.random.default_rng(5)
    q = np.concatenate([rng.integers(4096, 1 << 24, 4000), rng.integers(1 << 24, 1 << 27, 500)])
    q = np.concatenate([q, -q])
    got = _dequantize(q, w)
    ref = (q.astype(np.float64) * w).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_dequantize_exact_midpoints_single_width():
    """A single width and many q with q * w exactly a float midpoint in
    double: w = 2^-k makes every product exact."""
    w = 2.0 ** -20
    rng = np.random.default_rng(3)
    # q * 2^-20 is a float midpoint when q needs 25 significant bits
    q = (rng.integers(1 << 23, 1 << 24, 2000) * 2 + 1)
    q = q[q < 2 ** 31 - 1]
    got = _dequantize(q, w)
    ref = (q.astype(np.float64) * w).astype(np.float32)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
