"""CPU checks of the C ABI: the library loads, exports every function that
include/*.h declares, and its host-only logic (levels, bin widths, bounds)
agrees with the oracle.  No kernel is launched."""
import ctypes
import glob
import math
import os
import re

import numpy as np
import pytest

from oracle import bounds, grid
from paper_2401_05994_b300 import binding, build_ext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build_ext.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(mgard_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 20
    L = ctypes.CDLL(binding.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(binding.SIGNATURES), set(names) - set(binding.SIGNATURES)


def test_strerror_version():
    L = binding.lib()
    assert L.mgard_strerror(0) == b"ok"
    assert L.mgard_strerror(7).startswith(b"corrupt")
    assert L.mgard_version() >= 0x010000


@pytest.mark.parametrize("shape", [(129, 129), (513, 513, 513), (1, 33, 300), (7, 2), (1,), (5, 5, 5, 5)])
def test_levels_match_oracle(shape):
    assert binding.levels(shape) == grid.hierarchy(shape).L
    assert binding.levels(shape, 2) == grid.hierarchy(shape, 2).L


def test_bad_shapes_rejected():
    with pytest.raises(binding.MgardError) as e:
        binding.levels((3, 0))
    assert e.value.status == 2
    with pytest.raises(binding.MgardError):
        binding.levels((2, 2, 2, 2, 2))


@pytest.mark.parametrize("s", [math.inf, 0.0, 1.0, 0.5])
@pytest.mark.parametrize("shape", [(129, 129), (65, 65, 65), (33, 20, 47), (9, 6, 5, 7), (1000,), (300, 257)])
def test_bin_widths_match_oracle(shape, s):
    got = binding.bin_widths(shape, 0.37, s)
    exp = bounds.bin_widths(shape, 0.37, s)
    assert got.shape == exp.shape
    assert np.max(np.abs(got - exp) / exp) < 1e-12


def test_linf_width_of_the_benchmark_grid():
    """The L-infinity width of the 513^3 benchmark grid: the plan's per-level
    constants from unit solves against the oracle's dense evaluation, and
    the 1.39x gain over the earlier 1 + K_l bound."""
    shape = (513, 513, 513)
    got = binding.bin_widths(shape, 1.0, math.inf)
    exp = bounds.bin_widths(shape, 1.0, math.inf)
    assert np.max(np.abs(got - exp) / exp) < 1e-12
    h = grid.hierarchy(shape)
    old = 1.0 + sum(1.0 + bounds.K(h, l) for l in range(1, h.L + 1))
    assert 1.35 < got[0] / (2.0 * bounds.WIDTH_MARGIN / old) < 1.45


def test_bin_widths_large_axis_window():
    """Axes of more than 2048 coarse nodes evaluate the correction norm on
    windows near the ends and one interior row; the result must equal the
    oracle's exact dense evaluation."""
    got = binding.bin_widths((9001,), 1.0, math.inf)
    exp = bounds.bin_widths((9001,), 1.0, math.inf)
    assert np.max(np.abs(got - exp) / exp) < 1e-12


def test_compress_bound_is_an_upper_bound():
    n = 1000
    b = binding.compress_bound((n,))
    assert b > 8 * n
