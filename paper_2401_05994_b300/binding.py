"""Thin Python binding of the C ABI in ``include/mgard_b300.h``.

Argument marshalling only: every step runs in ``libmgard_b300.so``.  Device
arrays are ``torch.Tensor`` on CUDA (contiguous); host arrays are numpy
arrays or CPU tensors.  The functions carry the C names without the
``mgard_`` prefix.  If the compiled library is missing this module raises
on import of the library (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import struct
import math
import os
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgard_b300.so")

F32, F64 = 0, 1
ABS, REL = 0, 1
DICT = 4096
CHUNK = 1024
ESC = 0

_c_int64_p = ctypes.POINTER(ctypes.c_int64)
_c_double_p = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p

# name -> (restype, argtypes); mirrors include/mgard_b300.h
SIGNATURES = {
    "mgard_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "mgard_last_error": (ctypes.c_char_p, []),
    "mgard_version": (ctypes.c_uint32, []),
    "mgard_device_allocations": (ctypes.c_uint64, []),
    "mgard_levels": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "mgard_decompose": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_int, _vp]),
    "mgard_recompose": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_int, _vp]),
    "mgard_bin_widths": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, _c_double_p, ctypes.POINTER(ctypes.c_int)]),
    "mgard_norm": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, _c_double_p, _vp]),
    "mgard_error_norm": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, _c_double_p, _vp]),
    "mgard_quantize": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_int,
                                      _c_double_p, _vp, _vp, _vp, _vp]),
    "mgard_dequantize": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_int,
                                        _c_double_p, _vp, _vp]),
    "mgard_huffman_codebook": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "mgard_huffman_encode": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, _vp, _vp, ctypes.c_uint64, _vp, _vp,
                                            _vp, _vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64),
                                            ctypes.POINTER(ctypes.c_uint64), _vp]),
    "mgard_huffman_encode_noalloc": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, _vp, _vp, ctypes.c_uint64,
                                                    _vp, _vp, _vp, _vp, ctypes.c_uint64,
                                                    ctypes.POINTER(ctypes.c_uint64),
                                                    ctypes.POINTER(ctypes.c_uint64), _vp]),
    "mgard_huffman_decode": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp, _vp, _vp, _vp, ctypes.c_uint64, _vp,
                                            ctypes.c_uint64, _vp, _vp, _vp]),
    "mgard_compress_bound": (ctypes.c_size_t, [ctypes.c_int, _c_int64_p, ctypes.c_int]),
    "mgard_compress": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.POINTER(_vp),
                                      ctypes.POINTER(ctypes.c_size_t), ctypes.c_int, _vp]),
    "mgard_decompress": (ctypes.c_int, [_vp, ctypes.c_size_t, ctypes.POINTER(_vp), ctypes.c_int, _vp]),
    "mgard_decompress_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t),
                                              ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t),
                                              ctypes.POINTER(ctypes.c_int), ctypes.c_int, _vp]),
    "mgard_sizer_create": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_double,
                                          ctypes.POINTER(_vp), _vp]),
    "mgard_sizer_size": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t), _vp]),
    "mgard_sizer_features": (ctypes.c_int, [_vp, ctypes.c_double, _vp, _vp]),
    "mgard_sizer_compress": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_int, _vp,
                                            ctypes.POINTER(ctypes.c_size_t), _vp]),
    "mgard_sizer_free": (None, [_vp]),
    "mgard_mlp_init": (ctypes.c_int, [_vp, ctypes.c_uint64, _vp]),
    "mgard_mlp_set_norm": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "mgard_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "mgard_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, _vp, _vp]),
    "mgard_adam_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, ctypes.c_int, _vp]),
    "mgard_mlp_train": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_float, _vp, _vp]),
    "mgard_compress_to_ratio": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, _vp, ctypes.c_double, _c_double_p, _vp,
                                               ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_int),
                                               _vp]),
    "mgard_autotune": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_char_p,
                                      ctypes.c_size_t, _vp]),
    "mgard_compress_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(_c_int64_p), ctypes.c_int, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_int, ctypes.POINTER(_vp),
                                            ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t),
                                            ctypes.POINTER(ctypes.c_int), ctypes.c_int, _vp]),
    "mgard_refactor_bound": (ctypes.c_size_t, [ctypes.c_int, _c_int64_p, ctypes.c_int]),
    "mgard_refactor": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_int, _vp,
                                      ctypes.POINTER(ctypes.c_size_t), _vp]),
    "mgard_request": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.POINTER(ctypes.c_int32),
                                     ctypes.POINTER(ctypes.c_uint64), _c_double_p]),
    "mgard_reconstruct": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int32), _vp, _vp]),
    "mgard_qoi_representer": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, _vp, _vp]),
    "mgard_qoi_norm": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_double,
                                      _c_double_p, _vp]),
    "mgard_qoi_value": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _c_int64_p, ctypes.c_int, _c_double_p, _vp]),
    "mgard_compress_qoi": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, _vp, ctypes.c_double,
                                          ctypes.c_double, ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_size_t),
                                          ctypes.c_int, _c_double_p, _vp]),
    "mgard_region_plan": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_double, _vp, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int32)]),
    "mgard_region_exponents": (ctypes.c_int, [ctypes.c_int, _c_int64_p, ctypes.c_double, _vp, ctypes.c_int,
                                              _vp, _vp]),
    "mgard_compress_regions": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_double,
                                              _vp, ctypes.c_int, ctypes.POINTER(_vp),
                                              ctypes.POINTER(ctypes.c_size_t), ctypes.c_int, _vp]),
    "mgard_compress_ooc_bound": (ctypes.c_size_t, [ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_int64]),
    "mgard_compress_ooc": (ctypes.c_int, [_vp, ctypes.c_int, _c_int64_p, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int64, ctypes.POINTER(_vp),
                                          ctypes.POINTER(ctypes.c_size_t), ctypes.c_int, _vp]),
    "mgard_info": (ctypes.c_int, [_vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int), _c_int64_p,
                                  ctypes.POINTER(ctypes.c_int), _c_double_p, ctypes.POINTER(ctypes.c_int)]),
    "mgard_timing_enable": (None, [ctypes.c_int]),
    "mgard_timing_report": (ctypes.c_size_t, [ctypes.c_char_p, ctypes.c_size_t]),
    "mgard_free": (None, [_vp]),
    "mgard_release_plans": (None, []),
}

_lib = None


class MgardError(RuntimeError):
    def __init__(self, status: int, text: str):
        super().__init__(f"{text} (status {status})")
        self.status = status


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                               "`python -m paper_2401_05994_b300.build_ext`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int):
    if status != 0:
        L = lib()
        msg = L.mgard_strerror(status).decode()
        detail = L.mgard_last_error().decode()
        raise MgardError(status, f"{msg}: {detail}" if detail else msg)


def _shape(shape):
    shape = [int(s) for s in shape]
    return len(shape), (ctypes.c_int64 * len(shape))(*shape)


def _stream():
    if torch.cuda.is_available():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return None


def _dtype_code(dt) -> int:
    if dt in (torch.float32, np.float32, np.dtype(np.float32)):
        return F32
    if dt in (torch.float64, np.float64, np.dtype(np.float64)):
        return F64
    raise TypeError(f"unsupported dtype {dt}")


def _ptr(x):
    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(type(x))


def _require_cuda(t):
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("a CUDA tensor is required")


# ---- low level --------------------------------------------------------------

def levels(shape, max_levels: int = -1) -> int:
    nd, sh = _shape(shape)
    out = ctypes.c_int()
    _check(lib().mgard_levels(nd, sh, max_levels, ctypes.byref(out)))
    return out.value


def decompose(t: torch.Tensor, max_levels: int = -1) -> torch.Tensor:
    _require_cuda(t)
    nd, sh = _shape(t.shape)
    _check(lib().mgard_decompose(_ptr(t), nd, sh, _dtype_code(t.dtype), max_levels, _stream()))
    return t


def recompose(t: torch.Tensor, max_levels: int = -1) -> torch.Tensor:
    _require_cuda(t)
    nd, sh = _shape(t.shape)
    _check(lib().mgard_recompose(_ptr(t), nd, sh, _dtype_code(t.dtype), max_levels, _stream()))
    return t


def bin_widths(shape, tol_abs: float, s: float = math.inf, max_levels: int = -1) -> np.ndarray:
    nd, sh = _shape(shape)
    L = levels(shape, max_levels)
    w = np.zeros(L + 1)
    nl = ctypes.c_int()
    _check(lib().mgard_bin_widths(nd, sh, max_levels, tol_abs, s,
                                  w.ctypes.data_as(_c_double_p), ctypes.byref(nl)))
    return w


def norm(t: torch.Tensor, s: float = math.inf, max_levels: int = -1) -> float:
    _require_cuda(t)
    nd, sh = _shape(t.shape)
    out = ctypes.c_double()
    _check(lib().mgard_norm(_ptr(t), nd, sh, _dtype_code(t.dtype), max_levels, s,
                            ctypes.byref(out), _stream()))
    return out.value


def error_norm(a: torch.Tensor, b: torch.Tensor, s: float = math.inf, max_levels: int = -1) -> float:
    _require_cuda(a)
    _require_cuda(b)
    if a.shape != b.shape or a.dtype != b.dtype:
        raise ValueError("shape/dtype mismatch")
    nd, sh = _shape(a.shape)
    out = ctypes.c_double()
    _check(lib().mgard_error_norm(_ptr(a), _ptr(b), nd, sh, _dtype_code(a.dtype), max_levels, s,
                                  ctypes.byref(out), _stream()))
    return out.value


def quantize(coeffs: torch.Tensor, widths, max_levels: int = -1):
    """Returns (symbols uint16, escapes int32 indexed by symbol position,
    histogram int64) as CUDA tensors."""
    _require_cuda(coeffs)
    nd, sh = _shape(coeffs.shape)
    n = coeffs.numel()
    dev = coeffs.device
    sym = torch.empty(n, dtype=torch.uint16, device=dev)
    esc = torch.zeros(n, dtype=torch.int32, device=dev)
    hist = torch.empty(DICT, dtype=torch.int64, device=dev)
    w = np.ascontiguousarray(widths, dtype=np.float64)
    _check(lib().mgard_quantize(_ptr(coeffs), nd, sh, _dtype_code(coeffs.dtype), max_levels,
                                w.ctypes.data_as(_c_double_p), _ptr(sym), _ptr(esc), _ptr(hist),
                                _stream()))
    return sym, esc, hist


def dequantize(sym: torch.Tensor, esc: torch.Tensor, shape, dtype, widths,
               max_levels: int = -1, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    _require_cuda(sym)
    if out is None:
        out = torch.zeros(tuple(shape), dtype=dtype, device=sym.device)
    nd, sh = _shape(shape)
    w = np.ascontiguousarray(widths, dtype=np.float64)
    _check(lib().mgard_dequantize(_ptr(sym), _ptr(esc), nd, sh, _dtype_code(out.dtype), max_levels,
                                  w.ctypes.data_as(_c_double_p), _ptr(out), _stream()))
    return out


def huffman_codebook(hist: torch.Tensor):
    """Code lengths (uint8) and canonical codes (int32 view of uint32)."""
    _require_cuda(hist)
    lengths = torch.empty(DICT, dtype=torch.uint8, device=hist.device)
    codes = torch.empty(DICT, dtype=torch.int32, device=hist.device)
    _check(lib().mgard_huffman_codebook(_ptr(hist.to(torch.int64).contiguous()), _ptr(lengths),
                                        _ptr(codes), _stream()))
    return lengths, codes


def huffman_encode(sym: torch.Tensor, lengths: torch.Tensor, esc: torch.Tensor):
    """Returns (words int32 view of uint32, word_off int64, esc_off int64,
    sub_off uint16 [nchunks, 6], outliers int32)."""
    _require_cuda(sym)
    n = sym.numel()
    nchunks = (n + CHUNK - 1) // CHUNK
    dev = sym.device
    word_off = torch.empty(max(nchunks, 1), dtype=torch.int64, device=dev)
    esc_off = torch.empty(max(nchunks, 1), dtype=torch.int64, device=dev)
    sub_off = torch.zeros((max(nchunks, 1), 6), dtype=torch.uint16, device=dev)
    cap_w = n + nchunks + 1
    words = torch.empty(cap_w, dtype=torch.int32, device=dev)
    outl = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    nw = ctypes.c_uint64()
    no = ctypes.c_uint64()
    _check(lib().mgard_huffman_encode(_ptr(sym), n, _ptr(lengths), _ptr(esc), _ptr(words), cap_w,
                                      _ptr(word_off), _ptr(esc_off), _ptr(sub_off), _ptr(outl),
                                      max(n, 1), ctypes.byref(nw), ctypes.byref(no), _stream()))
    return (words[:nw.value], word_off[:nchunks], esc_off[:nchunks], sub_off[:nchunks],
            outl[:no.value])


def huffman_decode(words, word_off, esc_off, sub_off, lengths, n: int, outliers):
    _require_cuda(words)
    dev = words.device
    sym = torch.empty(max(n, 1), dtype=torch.uint16, device=dev)
    esc = torch.zeros(max(n, 1), dtype=torch.int32, device=dev)
    nout = outliers.numel()
    outliers = outliers if nout else torch.zeros(1, dtype=torch.int32, device=dev)
    _check(lib().mgard_huffman_decode(_ptr(words), words.numel(), _ptr(word_off), _ptr(esc_off),
                                      _ptr(sub_off), _ptr(lengths), n, _ptr(outliers), nout,
                                      _ptr(sym), _ptr(esc), _stream()))
    return sym[:n], esc[:n]


def timing_enable(on: bool = True):
    lib().mgard_timing_enable(1 if on else 0)


def timing_report() -> dict:
    """{kernel: (launches, total_ms)} of the traced launches (clears them)."""
    L = lib()
    need = L.mgard_timing_report(None, 0)
    buf = ctypes.create_string_buffer(max(need, 1) + 4096)
    L.mgard_timing_report(buf, len(buf))
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms = line.split()
        out[name] = (int(n), float(ms))
    return out


# ---- high level -------------------------------------------------------------

def compress_bound(shape, dtype=torch.float32) -> int:
    nd, sh = _shape(shape)
    return int(lib().mgard_compress_bound(nd, sh, _dtype_code(dtype)))


def compress(field, tol: float, s: float = math.inf, mode: int = REL, out=None):
    """Compress a CUDA tensor (result: CUDA uint8 tensor) or a host array
    (numpy / CPU tensor; result: numpy uint8 array).  ``out`` may supply a
    preallocated buffer of the same kind, at least ``compress_bound`` bytes."""
    host = not (isinstance(field, torch.Tensor) and field.is_cuda)
    if isinstance(field, torch.Tensor) and host:
        field = field.numpy()
    nd, sh = _shape(field.shape)
    dt = _dtype_code(field.dtype)
    if out is None:
        bound = compress_bound(field.shape, field.dtype)
        out = np.empty(bound, np.uint8) if host else torch.empty(bound, dtype=torch.uint8,
                                                                 device=field.device)
    nbytes = ctypes.c_size_t(out.nbytes if isinstance(out, np.ndarray) else out.numel())
    p = ctypes.c_void_p(_ptr(out).value)
    _check(lib().mgard_compress(_ptr(field), nd, sh, dt, float(tol), float(s), int(mode),
                                ctypes.byref(p), ctypes.byref(nbytes), 1, _stream()))
    return out[:nbytes.value]


def _weights(g: torch.Tensor, shape) -> torch.Tensor:
    if not (isinstance(g, torch.Tensor) and g.is_cuda and g.dtype == torch.float64):
        raise TypeError("QoI weights must be a CUDA float64 tensor")
    if tuple(g.shape) != tuple(shape):
        raise ValueError("QoI weights must have the field's shape")
    return g.contiguous()


def qoi_representer(g: torch.Tensor) -> torch.Tensor:
    """r = M_L^{-1} g on the grid of ``g`` (mgard_qoi_representer)."""
    g = _weights(g, g.shape)
    r = torch.empty_like(g)
    nd, sh = _shape(g.shape)
    _check(lib().mgard_qoi_representer(_ptr(g), nd, sh, _ptr(r), _stream()))
    return r


def qoi_norm(g: torch.Tensor, s: float, max_levels: int = -1) -> float:
    """Dual norm ||Q||_{-s} of the QoI with weights ``g`` (||g||_1 for s = inf)."""
    g = _weights(g, g.shape)
    nd, sh = _shape(g.shape)
    out = ctypes.c_double()
    _check(lib().mgard_qoi_norm(_ptr(g), nd, sh, int(max_levels), float(s), ctypes.byref(out), _stream()))
    return out.value


def qoi_value(field: torch.Tensor, g: torch.Tensor) -> float:
    """Q(field) = sum g * field in FP64 (mgard_qoi_value)."""
    g = _weights(g, field.shape)
    field = field.contiguous()
    nd, sh = _shape(field.shape)
    out = ctypes.c_double()
    _check(lib().mgard_qoi_value(_ptr(field), _ptr(g), nd, sh, _dtype_code(field.dtype),
                                 ctypes.byref(out), _stream()))
    return out.value


def compress_qoi(field: torch.Tensor, g: torch.Tensor, tol_qoi: float, s: float, out=None):
    """Compress a CUDA tensor so that the QoI's error stays within ``tol_qoi``
    (mgard_compress_qoi).  Returns ``(bytes, tol_used)``."""
    g = _weights(g, field.shape)
    nd, sh = _shape(field.shape)
    if out is None:
        out = torch.empty(compress_bound(field.shape, field.dtype), dtype=torch.uint8, device=field.device)
    nbytes = ctypes.c_size_t(out.numel())
    p = ctypes.c_void_p(_ptr(out).value)
    tol_used = ctypes.c_double()
    _check(lib().mgard_compress_qoi(_ptr(field), nd, sh, _dtype_code(field.dtype), _ptr(g), float(tol_qoi),
                                    float(s), ctypes.byref(p), ctypes.byref(nbytes), 1,
                                    ctypes.byref(tol_used), _stream()))
    return out[:nbytes.value], tol_used.value


class Region(ctypes.Structure):
    """mgard_region: inclusive index box (axes as passed) and its tolerance."""
    _fields_ = [("lo", ctypes.c_int64 * 4), ("hi", ctypes.c_int64 * 4), ("tol", ctypes.c_double)]


def _regions(regions):
    """[(lo, hi, tol), ...] -> ctypes array of mgard_region."""
    arr = (Region * max(1, len(regions)))()
    for r, (lo, hi, tol) in enumerate(regions):
        for d in range(len(lo)):
            arr[r].lo[d] = int(lo[d])
            arr[r].hi[d] = int(hi[d])
        arr[r].tol = float(tol)
    return arr


def region_plan(shape, tol: float, regions):
    """(rho, [k_r]) of mgard_region_plan."""
    nd, sh = _shape(shape)
    arr = _regions(regions)
    rho = ctypes.c_int()
    k = (ctypes.c_int32 * max(1, len(regions)))()
    _check(lib().mgard_region_plan(nd, sh, float(tol), ctypes.cast(arr, _vp), len(regions),
                                   ctypes.byref(rho), k))
    return rho.value, [int(k[i]) for i in range(len(regions))]


def region_exponents(shape, tol: float, regions, device="cuda") -> torch.Tensor:
    """Width exponent of every node (CUDA uint8 tensor of ``shape``)."""
    nd, sh = _shape(shape)
    arr = _regions(regions)
    out = torch.empty(tuple(shape), dtype=torch.uint8, device=device)
    _check(lib().mgard_region_exponents(nd, sh, float(tol), ctypes.cast(arr, _vp), len(regions),
                                        _ptr(out), _stream()))
    return out


def compress_regions(field: torch.Tensor, tol: float, regions, out=None):
    """Region-adaptive compression of a CUDA tensor (mgard_compress_regions):
    background absolute L-infinity tolerance ``tol``, boxes ``[(lo, hi, tol_r)]``."""
    nd, sh = _shape(field.shape)
    arr = _regions(regions)
    if out is None:
        out = torch.empty(compress_bound(field.shape, field.dtype) + 1024, dtype=torch.uint8,
                          device=field.device)
    nbytes = ctypes.c_size_t(out.numel())
    p = ctypes.c_void_p(_ptr(out).value)
    _check(lib().mgard_compress_regions(_ptr(field), nd, sh, _dtype_code(field.dtype), float(tol),
                                        ctypes.cast(arr, _vp), len(regions), ctypes.byref(p),
                                        ctypes.byref(nbytes), 1, _stream()))
    return out[:nbytes.value]


def compress_ooc_bound(shape, dtype, nblocks: int) -> int:
    nd, sh = _shape(shape)
    return int(lib().mgard_compress_ooc_bound(nd, sh, _dtype_code(dtype), int(nblocks)))


def compress_ooc(field, tol: float, nblocks: int, mode: int = ABS, out=None):
    """Out-of-core compression of a host array (numpy or CPU tensor, pinned
    for overlapped copies) in ``nblocks`` blocks along the first axis
    (mgard_compress_ooc).  ``out``: a host uint8 buffer (numpy or CPU tensor)
    of at least ``compress_ooc_bound`` bytes; returns the used prefix."""
    if isinstance(field, torch.Tensor):
        if field.is_cuda:
            raise TypeError("out-of-core compression takes a host field")
        dtype = field.dtype
    else:
        dtype = field.dtype
    nd, sh = _shape(field.shape)
    if out is None:
        out = np.empty(compress_ooc_bound(field.shape, dtype, nblocks), np.uint8)
    nbytes = ctypes.c_size_t(out.nbytes if isinstance(out, np.ndarray) else out.numel())
    p = ctypes.c_void_p(_ptr(out).value)
    _check(lib().mgard_compress_ooc(_ptr(field), nd, sh, _dtype_code(dtype), float(tol), int(mode),
                                    int(nblocks), ctypes.byref(p), ctypes.byref(nbytes), 1, _stream()))
    return out[:nbytes.value]


OOC_HEADER_FMT = "<8s4I4qddIIQ"


def ooc_blocks(buf) -> list:
    """(offset, end) of every block's buffer inside an out-of-core buffer."""
    raw = bytes(buf[:4096].tolist() if isinstance(buf, torch.Tensor) else buf[:4096])
    head = struct.unpack_from(OOC_HEADER_FMT, raw)
    nb = head[4]
    size = struct.calcsize(OOC_HEADER_FMT)
    allb = bytes(buf[:size + 8 * (nb + 1)].tolist() if isinstance(buf, torch.Tensor)
                 else buf[:size + 8 * (nb + 1)])
    offs = struct.unpack_from(f"<{nb + 1}Q", allb, size)
    return [(offs[b], offs[b + 1]) for b in range(nb)]


BATCH_GRAPH = 1
BATCH_AUTOTUNE = 2
BATCH_PERSISTENT = 8


def autotune(shape, dtype=torch.float32) -> str:
    """Tune the row kernels' launch shapes for ``shape`` (mgard_autotune);
    returns the tuner's report."""
    nd, sh = _shape(shape)
    buf = ctypes.create_string_buffer(1 << 16)
    _check(lib().mgard_autotune(nd, sh, _dtype_code(dtype), buf, len(buf), _stream()))
    return buf.value.decode()


def compress_batch(fields, tol: float, s: float = math.inf, mode: int = REL, outs=None,
                   graph: bool = False, check: bool = True, autotune: bool = False,
                   persistent: bool = False):
    """Compress a list of CUDA tensors in one call (mgard_compress_batch).

    ``outs``: list of CUDA uint8 tensors (default: ``compress_bound`` bytes
    each).  Returns ``(views, sizes, statuses)``: the compressed bytes of
    every field (views into ``outs``), their sizes and per-field status
    codes.  With ``check`` a failing field raises."""
    n = len(fields)
    if n == 0:
        return [], [], []
    dt = _dtype_code(fields[0].dtype)
    for f in fields:
        _require_cuda(f)
        if _dtype_code(f.dtype) != dt:
            raise ValueError("all fields of a batch share one dtype")
    if outs is None:
        outs = [torch.empty(compress_bound(f.shape, f.dtype), dtype=torch.uint8, device=f.device)
                for f in fields]
    shapes = [_shape(f.shape) for f in fields]
    fptr = (_vp * n)(*[f.data_ptr() for f in fields])
    optr = (_vp * n)(*[o.data_ptr() for o in outs])
    nds = (ctypes.c_int * n)(*[sh[0] for sh in shapes])
    shp = (_c_int64_p * n)(*[ctypes.cast(sh[1], _c_int64_p) for sh in shapes])
    caps = (ctypes.c_size_t * n)(*[o.numel() for o in outs])
    sizes = (ctypes.c_size_t * n)()
    stats = (ctypes.c_int * n)()
    st = lib().mgard_compress_batch(n, fptr, nds, shp, dt, float(tol), float(s), int(mode), optr,
                                    caps, sizes, stats,
                                    (BATCH_GRAPH if graph else 0) | (BATCH_AUTOTUNE if autotune else 0)
                                    | (BATCH_PERSISTENT if persistent else 0),
                                    _stream())
    if check:
        _check(st)
    sizes = [int(x) for x in sizes]
    return [o[:min(z, o.numel())] for o, z in zip(outs, sizes)], sizes, [int(x) for x in stats]


def decompress_batch(bufs, outs=None, graph: bool = False, check: bool = True,
                     persistent: bool = False):
    """Decompress a list of CUDA uint8 tensors (mgard_decompress_batch).
    ``outs``: list of CUDA tensors of the fields' shapes and dtypes (default:
    allocated from the headers).  Returns ``(outs, statuses)``."""
    n = len(bufs)
    if n == 0:
        return [], []
    for b in bufs:
        _require_cuda(b)
    if outs is None:
        outs = []
        for b in bufs:
            m = info(b)
            outs.append(torch.empty(m["shape"], dtype=m["dtype"], device=b.device))
    iptr = (_vp * n)(*[b.data_ptr() for b in bufs])
    isz = (ctypes.c_size_t * n)(*[b.numel() for b in bufs])
    optr = (_vp * n)(*[o.data_ptr() for o in outs])
    ocap = (ctypes.c_size_t * n)(*[o.numel() * o.element_size() for o in outs])
    stats = (ctypes.c_int * n)()
    st = lib().mgard_decompress_batch(n, iptr, isz, optr, ocap, stats,
                                      (BATCH_GRAPH if graph else 0)
                                      | (BATCH_PERSISTENT if persistent else 0), _stream())
    if check:
        _check(st)
    return outs, [int(x) for x in stats]


# ---- ratio targeting and the tolerance predictor ----------------------------
NFEAT = 220
MLP_HIDDEN = 64
MLP_NTRAIN = MLP_HIDDEN * NFEAT + MLP_HIDDEN * MLP_HIDDEN + 3 * MLP_HIDDEN + 1
MLP_NPARAM = MLP_NTRAIN + 2 * NFEAT


class Sizer:
    """One decomposition of a CUDA field; exact compressed sizes, predictor
    features and the final compression at any tolerance (mgard_sizer_*).
    The field must not change while the sizer is open."""

    def __init__(self, field, s: float = math.inf):
        _require_cuda(field)
        self.field = field
        nd, sh = _shape(field.shape)
        h = _vp()
        _check(lib().mgard_sizer_create(field.data_ptr(), nd, sh, _dtype_code(field.dtype), float(s),
                                        ctypes.byref(h), _stream()))
        self.h = h

    def size(self, tol: float, mode: int = REL) -> int:
        b = ctypes.c_size_t()
        _check(lib().mgard_sizer_size(self.h, float(tol), int(mode), ctypes.byref(b), _stream()))
        return int(b.value)

    def features(self, target_ratio: float, out=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(NFEAT, dtype=torch.float32, device=self.field.device)
        _check(lib().mgard_sizer_features(self.h, float(target_ratio), out.data_ptr(), _stream()))
        return out

    def compress(self, tol: float, mode: int = REL, out=None):
        if out is None:
            out = torch.empty(compress_bound(self.field.shape, self.field.dtype), dtype=torch.uint8,
                              device=self.field.device)
        n = ctypes.c_size_t(out.numel())
        _check(lib().mgard_sizer_compress(self.h, float(tol), int(mode), out.data_ptr(),
                                          ctypes.byref(n), _stream()))
        return out[:n.value]

    def close(self):
        if self.h:
            lib().mgard_sizer_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def mlp_init(seed: int = 0, device="cuda") -> torch.Tensor:
    p = torch.empty(MLP_NPARAM, dtype=torch.float32, device=device)
    _check(lib().mgard_mlp_init(p.data_ptr(), int(seed), _stream()))
    return p


def mlp_set_norm(params: torch.Tensor, x: torch.Tensor):
    _check(lib().mgard_mlp_set_norm(params.data_ptr(), x.data_ptr(), x.shape[0], _stream()))


def mlp_forward(params: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    x = x.contiguous()
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    _check(lib().mgard_mlp_forward(params.data_ptr(), x.data_ptr(), x.shape[0], y.data_ptr(), _stream()))
    return y


def mlp_loss_grad(params: torch.Tensor, x: torch.Tensor, t: torch.Tensor):
    x, t = x.contiguous(), t.contiguous()
    g = torch.empty(MLP_NTRAIN, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _check(lib().mgard_mlp_loss_grad(params.data_ptr(), x.data_ptr(), t.data_ptr(), x.shape[0],
                                     g.data_ptr(), loss.data_ptr(), _stream()))
    return loss, g


def adam_step(params, grad, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(lib().mgard_adam_step(params.data_ptr(), grad.data_ptr(), m.data_ptr(), v.data_ptr(),
                                 grad.numel(), lr, beta1, beta2, eps, int(t), _stream()))


def mlp_train(params, m, v, x, t, steps: int, t0: int = 0, lr: float = 1e-3) -> torch.Tensor:
    x, t = x.contiguous(), t.contiguous()
    losses = torch.empty(max(steps, 1), dtype=torch.float32, device=x.device)
    _check(lib().mgard_mlp_train(params.data_ptr(), m.data_ptr(), v.data_ptr(), x.data_ptr(),
                                 t.data_ptr(), x.shape[0], int(steps), int(t0), float(lr),
                                 losses.data_ptr(), _stream()))
    return losses[:steps]


def compress_to_ratio(field, target_ratio: float, s: float = math.inf, params=None,
                      rel_err: float = 0.05, out=None):
    """Compress a CUDA field at the relative tolerance that reaches
    ``target_ratio`` within ``rel_err`` (mgard_compress_to_ratio).  Returns
    ``(buffer view, tol, passes)``."""
    _require_cuda(field)
    nd, sh = _shape(field.shape)
    if out is None:
        out = torch.empty(compress_bound(field.shape, field.dtype), dtype=torch.uint8, device=field.device)
    n = ctypes.c_size_t(out.numel())
    tol = ctypes.c_double()
    passes = ctypes.c_int()
    _check(lib().mgard_compress_to_ratio(field.data_ptr(), nd, sh, _dtype_code(field.dtype),
                                         float(target_ratio), float(s),
                                         params.data_ptr() if params is not None else None,
                                         float(rel_err), ctypes.byref(tol), out.data_ptr(),
                                         ctypes.byref(n), ctypes.byref(passes), _stream()))
    return out[:n.value], tol.value, passes.value


def info(buf):
    nd = ctypes.c_int()
    shape = (ctypes.c_int64 * 4)()
    dt = ctypes.c_int()
    tol_abs = ctypes.c_double()
    nl = ctypes.c_int()
    nbytes = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel()
    _check(lib().mgard_info(_ptr(buf), nbytes, ctypes.byref(nd), shape, ctypes.byref(dt),
                            ctypes.byref(tol_abs), ctypes.byref(nl)))
    return dict(shape=tuple(shape[i] for i in range(nd.value)),
                dtype=torch.float64 if dt.value == F64 else torch.float32,
                tol_abs=tol_abs.value, nlevels=nl.value)


def decompress(buf, out=None):
    """Inverse of :func:`compress` (same placement rules)."""
    meta = info(buf)
    host = isinstance(buf, np.ndarray)
    if out is None:
        if host:
            out = np.empty(meta["shape"], dtype=np.float64 if meta["dtype"] == torch.float64
                           else np.float32)
        else:
            out = torch.empty(meta["shape"], dtype=meta["dtype"], device=buf.device)
    nbytes = buf.nbytes if host else buf.numel()
    p = ctypes.c_void_p(_ptr(out).value)
    _check(lib().mgard_decompress(_ptr(buf), nbytes, ctypes.byref(p), 1, _stream()))
    return out


# -- refactoring (progressive retrieval) ------------------------------------
MDR_HEADER_FMT = "<8s6I4qdQ"
MDR_LEVEL_FMT = "<QQIiIId"
MDR_MAX_LEVELS = 64
MDR_HEADER_SIZE = (struct.calcsize(MDR_HEADER_FMT)
                   + (MDR_MAX_LEVELS + 1) * struct.calcsize(MDR_LEVEL_FMT))


def mdr_header(buf) -> dict:
    """Parsed header of a refactored buffer (device tensor or bytes); the
    raw header bytes are under "raw"."""
    raw = (buf[:MDR_HEADER_SIZE].cpu().numpy().tobytes() if isinstance(buf, torch.Tensor)
           else bytes(buf[:MDR_HEADER_SIZE]))
    f = struct.unpack_from(MDR_HEADER_FMT, raw, 0)
    h = dict(magic=f[0], version=f[1], dtype=f[2], ndim=f[3], nlevels=f[4], planes=f[5],
             shape=tuple(f[7:7 + f[3]]), max_abs=f[11], total_bytes=f[12], raw=raw)
    base = struct.calcsize(MDR_HEADER_FMT)
    size = struct.calcsize(MDR_LEVEL_FMT)
    h["levels"] = []
    for l in range(h["nlevels"]):
        c, off, words, e, nz, _, w = struct.unpack_from(MDR_LEVEL_FMT, raw, base + l * size)
        h["levels"].append(dict(count=c, offset=off, words=words, exponent=e, nonzero=bool(nz),
                                weight=w))
    return h


def refactor_bound(shape, planes: int = 32) -> int:
    nd, sh = _shape(shape)
    return int(lib().mgard_refactor_bound(nd, sh, planes))


def refactor(field: torch.Tensor, planes: int = 32):
    """MDRefactor of a CUDA tensor: (device uint8 buffer, parsed header)."""
    _require_cuda(field)
    nd, sh = _shape(field.shape)
    cap = refactor_bound(field.shape, planes)
    out = torch.empty(cap, dtype=torch.uint8, device=field.device)
    nbytes = ctypes.c_size_t(cap)
    _check(lib().mgard_refactor(_ptr(field.contiguous()), nd, sh, _dtype_code(field.dtype), planes,
                                _ptr(out), ctypes.byref(nbytes), _stream()))
    out = out[:nbytes.value]
    return out, mdr_header(out)


def request(header: dict, tol: float):
    """MDRequest: (planes per level, bytes of those planes, estimate)."""
    raw = ctypes.create_string_buffer(header["raw"], len(header["raw"]))
    n = header["nlevels"]
    P = (ctypes.c_int32 * n)()
    nb = ctypes.c_uint64()
    est = ctypes.c_double()
    st = lib().mgard_request(ctypes.cast(raw, ctypes.c_void_p), float(tol), P, ctypes.byref(nb),
                             ctypes.byref(est))
    if st not in (0, 8):   # MGARD_EBOUND still returns every plane
        _check(st)
    return list(P), nb.value, est.value


def reconstruct(buf: torch.Tensor, planes, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """MDReconstruct from a refactored device buffer with `planes` per level."""
    _require_cuda(buf)
    h = mdr_header(buf)
    dt = torch.float32 if h["dtype"] == 0 else torch.float64
    if out is None:
        out = torch.empty(h["shape"], dtype=dt, device=buf.device)
    P = (ctypes.c_int32 * len(planes))(*[int(p) for p in planes])
    _check(lib().mgard_reconstruct(_ptr(buf), P, _ptr(out), _stream()))
    return out
