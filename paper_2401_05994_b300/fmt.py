"""Parser of the compressed buffer layout documented in
include/mgard_format.h (reads bytes only; for inspection and tests)."""
import struct

import numpy as np

HEADER_FMT = "<8sIIII4qdddIIIIQQQQQQQQQQQQ"
HEADER_SIZE = struct.calcsize(HEADER_FMT)
FIELDS = ["magic", "version", "dtype", "ndim", "nlevels", "s0", "s1", "s2", "s3", "s", "tol",
          "tol_abs", "mode", "dict", "chunk", "reserved", "nsymbols", "nchunks", "nwords",
          "noutliers", "off_widths", "off_lengths", "off_word_off", "off_esc_off",
          "off_sub_off", "off_outliers", "off_words", "total_bytes"]


def parse(buf: bytes):
    h = dict(zip(FIELDS, struct.unpack_from(HEADER_FMT, buf, 0)))
    b = np.frombuffer(buf, dtype=np.uint8)
    L = h["nlevels"]
    sec = {}
    sec["widths"] = b[h["off_widths"]:h["off_widths"] + 8 * (L + 1)].view(np.float64)
    sec["lengths"] = b[h["off_lengths"]:h["off_lengths"] + h["dict"]].copy()
    n = h["nchunks"]
    sec["word_off"] = b[h["off_word_off"]:h["off_word_off"] + 8 * n].view(np.uint64)
    sec["esc_off"] = b[h["off_esc_off"]:h["off_esc_off"] + 8 * n].view(np.uint64)
    sec["sub_off"] = b[h["off_sub_off"]:h["off_sub_off"] + 12 * n].view(np.uint16).reshape(n, 6)
    sec["outliers"] = b[h["off_outliers"]:h["off_outliers"] + 4 * h["noutliers"]].view(np.int32)
    sec["words"] = b[h["off_words"]:h["off_words"] + 4 * h["nwords"]].view(np.uint32)
    return h, sec


def header(buf: bytes):
    return dict(zip(FIELDS, struct.unpack_from(HEADER_FMT, buf, 0)))
