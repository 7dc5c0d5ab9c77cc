"""Test helpers for the JPEG pipeline: a writer of baseline grayscale JPEGs
whose 8x8 blocks are flat, and a reader of JPEG frame headers.

The writer follows ITU-T T.81 (baseline sequential DCT, Huffman coded) for
the one case whose decoded pixels are known exactly without a decoder: every
block constant.  A block of value v has only a DC coefficient, 8 (v - 128)
(the forward DCT of a constant block), all quantisers are 1, and the inverse
DCT of a DC-only block is DC / 8 everywhere, so a conforming decoder
reproduces v exactly.  The stream carries its own Huffman tables (T.81
allows any): DC categories 0..11 get the 4-bit codes 0000..1011 and the AC
table holds only end-of-block, code 0.  No filter arithmetic here.
"""
from __future__ import annotations

import struct

import numpy as np


def _segment(marker: int, payload: bytes) -> bytes:
    return struct.pack(">HH", marker, len(payload) + 2) + payload


class _Bits:
    def __init__(self):
        self.out = bytearray()
        self.acc = 0
        self.n = 0

    def put(self, value: int, nbits: int):
        for i in range(nbits - 1, -1, -1):
            self.acc = (self.acc << 1) | ((value >> i) & 1)
            self.n += 1
            if self.n == 8:
                self.out.append(self.acc)
                if self.acc == 0xFF:        # byte stuffing (T.81 F.1.2.3)
                    self.out.append(0x00)
                self.acc, self.n = 0, 0

    def flush(self) -> bytes:
        if self.n:                          # pad with 1-bits
            self.put((1 << (8 - self.n)) - 1, 8 - self.n)
        return bytes(self.out)


def flat_gray_jpeg(blocks: np.ndarray, width: int | None = None,
                   height: int | None = None) -> bytes:
    """Baseline grayscale JPEG of a (by, bx) array of block values (uint8):
    the image is (8 by) x (8 bx) pixels, block (i, j) filled with blocks[i, j],
    or its top-left width x height pixels (the frame header then gives the
    smaller size, and a decoder drops the edge blocks' pixels beyond it,
    T.81 A.1.1); width > 8 (bx - 1) and height > 8 (by - 1)."""
    blocks = np.asarray(blocks, dtype=np.int64)
    by, bx = blocks.shape
    h = 8 * by if height is None else height
    w = 8 * bx if width is None else width
    if not (8 * (by - 1) < h <= 8 * by and 8 * (bx - 1) < w <= 8 * bx):
        raise ValueError("size does not match the block grid")
    out = bytearray(b"\xff\xd8")                                            # SOI
    out += _segment(0xFFDB, bytes([0x00]) + bytes([1] * 64))                # DQT: table 0, all 1
    out += _segment(0xFFC0, struct.pack(">BHHB", 8, h, w, 1) + bytes([1, 0x11, 0]))  # SOF0
    dc_bits = [0, 0, 0, 12] + [0] * 12                                       # 12 codes of length 4
    out += _segment(0xFFC4, bytes([0x00] + dc_bits + list(range(12))))      # DHT: DC table 0
    ac_bits = [1] + [0] * 15                                                 # 1 code of length 1
    out += _segment(0xFFC4, bytes([0x10] + ac_bits + [0x00]))               # DHT: AC table 0 (EOB)
    out += _segment(0xFFDA, bytes([1, 1, 0x00, 0, 63, 0]))                  # SOS
    bits = _Bits()
    pred = 0
    for v in blocks.reshape(-1):                                            # raster order of blocks
        dc = 8 * (int(v) - 128)
        diff = dc - pred
        pred = dc
        size = 0 if diff == 0 else abs(diff).bit_length()                   # category (T.81 F.1.2.1)
        bits.put(size, 4)                                                   # its code
        if size:
            bits.put(diff if diff > 0 else diff + (1 << size) - 1, size)    # additional bits
        bits.put(0, 1)                                                      # EOB
    out += bits.flush()
    out += b"\xff\xd9"                                                      # EOI
    return bytes(out)


def flat_gray_jpeg_progressive(blocks: np.ndarray, width: int | None = None,
                               height: int | None = None) -> bytes:
    """The image of flat_gray_jpeg(blocks, width, height) as a progressive
    JPEG (T.81 Annex G, SOF2): a DC first scan (Ss = Se = 0, no successive
    approximation) coding the same DC differences as the baseline stream,
    then one AC scan (Ss = 1, Se = 63) in which every block is a lone
    end-of-band (EOB0: an end-of-band run of one block).  Its decoded pixels
    are the same known image."""
    blocks = np.asarray(blocks, dtype=np.int64)
    by, bx = blocks.shape
    h = 8 * by if height is None else height
    w = 8 * bx if width is None else width
    if not (8 * (by - 1) < h <= 8 * by and 8 * (bx - 1) < w <= 8 * bx):
        raise ValueError("size does not match the block grid")
    out = bytearray(b"\xff\xd8")                                            # SOI
    out += _segment(0xFFDB, bytes([0x00]) + bytes([1] * 64))                # DQT: table 0, all 1
    out += _segment(0xFFC2, struct.pack(">BHHB", 8, h, w, 1) + bytes([1, 0x11, 0]))  # SOF2
    dc_bits = [0, 0, 0, 12] + [0] * 12
    out += _segment(0xFFC4, bytes([0x00] + dc_bits + list(range(12))))      # DHT: DC table 0
    ac_bits = [1] + [0] * 15
    out += _segment(0xFFC4, bytes([0x10] + ac_bits + [0x00]))               # DHT: AC table 0 (EOB0)
    # DC first scan: component 1, DC table 0; Ss = 0, Se = 0, Ah = Al = 0
    out += _segment(0xFFDA, bytes([1, 1, 0x00, 0, 0, 0]))
    bits = _Bits()
    pred = 0
    for v in blocks.reshape(-1):
        dc = 8 * (int(v) - 128)
        diff = dc - pred
        pred = dc
        size = 0 if diff == 0 else abs(diff).bit_length()
        bits.put(size, 4)
        if size:
            bits.put(diff if diff > 0 else diff + (1 << size) - 1, size)
    out += bits.flush()
    # AC scan: component 1, AC table 0; Ss = 1, Se = 63, Ah = Al = 0; a
    # one-component scan covers the component's ceil(w/8) x ceil(h/8) blocks
    out += _segment(0xFFDA, bytes([1, 1, 0x00, 1, 63, 0]))
    bits = _Bits()
    for _ in range(((w + 7) // 8) * ((h + 7) // 8)):
        bits.put(0, 1)                                                      # EOB0
    out += bits.flush()
    out += b"\xff\xd9"                                                      # EOI
    return bytes(out)


def flat_gray_image(blocks: np.ndarray, width: int | None = None,
                    height: int | None = None) -> np.ndarray:
    """The grayscale image flat_gray_jpeg(blocks, width, height) encodes."""
    img = np.kron(np.asarray(blocks, dtype=np.uint8), np.ones((8, 8), dtype=np.uint8))
    return img[:height, :width]


def frame_header(data: bytes) -> dict:
    """Width, height, components and their sampling factors from the first
    SOF marker; checks that the stream starts with SOI and ends with EOI."""
    assert data[:2] == b"\xff\xd8", "no SOI"
    assert data[-2:] == b"\xff\xd9", "no EOI"
    i = 2
    while i + 4 <= len(data):
        assert data[i] == 0xFF, f"marker expected at {i}"
        marker = data[i + 1]
        if marker == 0xFF:          # fill byte
            i += 1
            continue
        length = struct.unpack(">H", data[i + 2:i + 4])[0]
        if marker in (0xC0, 0xC1, 0xC2):
            p, h, w, nf = struct.unpack(">BHHB", data[i + 4:i + 10])
            comps = [(data[i + 10 + 3 * k], data[i + 11 + 3 * k] >> 4, data[i + 11 + 3 * k] & 15)
                     for k in range(nf)]
            return {"precision": p, "width": w, "height": h, "components": nf,
                    "sampling": [(hs, vs) for _, hs, vs in comps], "sof": marker}
        if marker == 0xDA:
            break
        i += 2 + length
    raise AssertionError("no SOF marker before the scan")
