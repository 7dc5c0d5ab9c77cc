"""The JPEG pipeline library (include/oilpaint_jpeg.h) builds, loads and
exports every declared entry point, its argument checks that come before any
CUDA call behave, and the test JPEG writer produces well-formed streams.  No
GPU needed."""
import os
import re

import numpy as np
import pytest

from paper_1405_1020_gb300 import jpeg as J
from paper_1405_1020_gb300.binding import OP_E_INVALID, OP_OK
from paper_1405_1020_gb300.csrc import build as cbuild
from tests.jpeg_fixture import (flat_gray_image, flat_gray_jpeg, flat_gray_jpeg_progressive,
                                frame_header)

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "oilpaint_jpeg.h")


def declared():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return sorted(set(re.findall(r"\b(op_jpeg_[a-z_]+)\s*\(", text)))


def header_constants():
    text = open(HEADER).read()
    return {m.group(1): int(m.group(2))
            for m in re.finditer(r"#define\s+(OP_\w+)\s+\(?(-?\d+)\)?", text)}


@pytest.fixture(scope="module")
def lib():
    cbuild.build()
    if cbuild.build_jpeg() is None:
        pytest.skip("nvJPEG is not in this CUDA toolkit")
    return J.load()


def test_header_and_binding_agree():
    assert sorted(J.EXPORTS) == declared()
    consts = header_constants()
    for name in ("OP_E_CODEC", "OP_E_NOSPACE", "OP_JPEG_CSS_444", "OP_JPEG_CSS_422",
                 "OP_JPEG_CSS_420", "OP_JPEG_MAX_BATCH"):
        assert consts[name] == getattr(J, name), name


def test_every_declared_symbol_is_exported(lib):
    for name in declared():
        assert hasattr(lib, name), name


def test_null_handles(lib):
    import ctypes
    n = ctypes.c_size_t()
    w = ctypes.c_uint32()
    assert J.op_jpeg_info(None, b"\xff\xd8", w, None, None) == OP_E_INVALID
    assert J.op_jpeg_decode(None, b"\xff\xd8", 1 << 20, 30) == OP_E_INVALID
    assert J.op_jpeg_encode_bound(None, 10, 10, 90, 0, n) == OP_E_INVALID
    assert J.op_jpeg_encode(None, 1 << 20, 10, 10, 30, 90, 0, None, 0, n) == OP_E_INVALID
    assert J.op_jpeg_filter(None, b"\xff\xd8", 2, 20, 0, 90, 0, None, 0, n) == OP_E_INVALID
    assert J.op_jpeg_filter_file(None, "a.jpg", "b.jpg", 2, 20, 0, 90, 0) == OP_E_INVALID
    arr = lambda t: (t * 1)()  # noqa: E731
    assert J.op_jpeg_filter_batch(None, [b"\xff\xd8"], 2, 20, 0, 90, 0, arr(ctypes.c_void_p),
                                  arr(ctypes.c_size_t), arr(ctypes.c_size_t),
                                  arr(ctypes.c_int)) == OP_E_INVALID
    assert J.op_jpeg_last_timing(None, J.op_jpeg_timing_t()) == OP_E_INVALID
    assert J.op_jpeg_destroy(None) == OP_OK


def test_status_strings():
    assert "nvJPEG" in J.status_string(J.OP_E_CODEC)
    assert "small" in J.status_string(J.OP_E_NOSPACE)


def test_flat_gray_writer():
    rng = np.random.default_rng(0)
    blocks = rng.integers(0, 256, size=(5, 7)).astype(np.uint8)
    blocks[0, 0], blocks[0, 1] = 0, 255
    data = flat_gray_jpeg(blocks)
    hdr = frame_header(data)
    assert hdr == {"precision": 8, "width": 56, "height": 40, "components": 1,
                   "sampling": [(1, 1)], "sof": 0xC0}
    # entropy-coded data: every 0xFF is stuffed, so the only markers left are SOS's and EOI
    scan = data[data.index(b"\xff\xda") + 2 + 8:-2]
    for i in np.flatnonzero(np.frombuffer(scan, dtype=np.uint8) == 0xFF):
        assert scan[i + 1] == 0x00
    img = flat_gray_image(blocks)
    assert img.shape == (40, 56) and img[8 * 4 + 3, 8 * 6 + 5] == blocks[4, 6]


def test_flat_gray_writer_ragged_size():
    blocks = np.arange(12, dtype=np.uint8).reshape(3, 4) * 20
    data = flat_gray_jpeg(blocks, 29, 17)
    hdr = frame_header(data)
    assert (hdr["width"], hdr["height"]) == (29, 17)
    img = flat_gray_image(blocks, 29, 17)
    assert img.shape == (17, 29) and img[16, 28] == blocks[2, 3]
    # the entropy-coded data is that of the whole block grid either way
    full = flat_gray_jpeg(blocks)
    assert data[data.index(b"\xff\xda"):] == full[full.index(b"\xff\xda"):]
    with pytest.raises(ValueError):
        flat_gray_jpeg(blocks, 24, 17)


def _segments(data: bytes):
    """(marker, payload) of every marker segment before EOI, entropy-coded
    data skipped (T.81 B.1.1.2: 0xFF00 is a stuffed byte, not a marker)."""
    out, i = [], 2
    while i < len(data) - 2:
        assert data[i] == 0xFF
        marker = data[i + 1]
        n = int.from_bytes(data[i + 2:i + 4], "big")
        out.append((marker, data[i + 4:i + 2 + n]))
        i += 2 + n
        if marker == 0xDA:                      # skip the scan's entropy-coded data
            while not (data[i] == 0xFF and data[i + 1] != 0x00):
                i += 1
    return out


def test_flat_gray_progressive_writer():
    blocks = np.arange(35, dtype=np.uint8).reshape(5, 7) * 7
    data = flat_gray_jpeg_progressive(blocks, 53, 37)
    hdr = frame_header(data)
    assert hdr["sof"] == 0xC2 and (hdr["width"], hdr["height"]) == (53, 37)
    scans = [p for m, p in _segments(data) if m == 0xDA]
    # a DC first scan, then one AC scan over bands 1..63, one component each
    assert [tuple(p[-3:]) for p in scans] == [(0, 0, 0), (1, 63, 0)]
    assert all(p[0] == 1 for p in scans)
    # the AC scan codes one EOB0 (a single 0 bit) per block, padded with 1s
    ac = data[data.rindex(b"\xff\xda") + 2 + 8:-2]
    assert ac == b"\x00" * 4 + bytes([0b00011111])
    assert data.count(b"\xff\xda") == 2       # two scans, no third
    with pytest.raises(ValueError):
        flat_gray_jpeg_progressive(blocks, 48, 37)
