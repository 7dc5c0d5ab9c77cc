"""CPU oracles for the histogram oil-paint filter -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  The product
path (``paper_1405_1020_gb300``) never does, and shares no code with it.

* ``oilpaint`` / ``oilpaint_rows`` / ``oilpaint_pixels``: the plain C
  brute-force oracle (``oilpaint_ref.c``), threaded over rows;
* ``oilpaint_numpy`` (module ``oilpaint_np``): the independent NumPy
  integral-image oracle.

Both follow section 4 of Mukherjee, arXiv 1405.1020 (histogram of intensity
levels per (2r+1)^2 window; most frequent level, lowest on a tie; truncated
channel means of that level), with out-of-image neighbours skipped.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build
from . import oilpaint_np  # noqa: F401  (the NumPy oracle module)
from .oilpaint_np import LEVEL_INTDIV3, LEVEL_PAPER, level_map  # noqa: F401

# mode bit of the C oracle: the section-4 listing as printed (interior pixels
# only, white excluded from the argmax, no write when no level below L occurs)
LITERAL = 2
from .oilpaint_np import oilpaint_buffer as oilpaint_numpy  # noqa: F401

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        u32 = ctypes.c_uint32
        lib.orc_oilpaint_rows.argtypes = [u8p, u8p, u32, u32, u32, u32, ctypes.c_int32, u32, u32,
                                          u32, u32, ctypes.c_int]
        lib.orc_oilpaint_rows.restype = ctypes.c_int
        lib.orc_oilpaint_pixels.argtypes = [u8p, u32, u32, u32, u32, ctypes.c_int32, u32, u32,
                                            u32p, u32p, u32, u8p]
        lib.orc_oilpaint_pixels.restype = ctypes.c_int
        lib.orc_level_of_sum.argtypes = [u32, u32, u32]
        lib.orc_level_of_sum.restype = u32
        lib.orc_num_cpus.argtypes = []
        lib.orc_num_cpus.restype = ctypes.c_int
        _lib = lib
    return _lib


def _u8(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def num_cpus() -> int:
    return int(_load().orc_num_cpus())


def level_of_sum(s: int, levels: int, mode: int = LEVEL_PAPER) -> int:
    return int(_load().orc_level_of_sum(s, levels, mode))


def oilpaint_rows(buf: np.ndarray, width: int, height: int, stride: int, bpp: int, radius: int,
                  levels: int, y_begin: int, y_end: int, mode: int = LEVEL_PAPER,
                  threads: int = 0, out: np.ndarray | None = None) -> np.ndarray:
    """Rows [y_begin, y_end) of the filtered image into `out` (a copy of
    nothing: a zero buffer of buf's size unless given).  Row padding and rows
    outside the range are left as they are in `out`."""
    src = np.ascontiguousarray(buf, dtype=np.uint8).reshape(-1)
    if src.size < height * stride:
        raise ValueError("buffer too small")
    if out is None:
        out = np.zeros_like(src)
    if not (out.flags["C_CONTIGUOUS"] and out.dtype == np.uint8 and out.size >= height * stride):
        raise ValueError("out must be a contiguous uint8 buffer of at least height*stride bytes")
    rc = _load().orc_oilpaint_rows(_u8(src), _u8(out), width, height, stride, bpp, radius, levels,
                                   mode, y_begin, y_end, threads)
    if rc != 0:
        raise ValueError(f"oracle rejected arguments (status {rc})")
    return out


def oilpaint(buf: np.ndarray, width: int, height: int, stride: int, bpp: int, radius: int,
             levels: int, mode: int = LEVEL_PAPER, threads: int = 0,
             out: np.ndarray | None = None) -> np.ndarray:
    """Whole image; see ``oilpaint_rows``."""
    return oilpaint_rows(buf, width, height, stride, bpp, radius, levels, 0, height, mode,
                         threads, out)


def oilpaint_pixels(buf: np.ndarray, width: int, height: int, stride: int, bpp: int, radius: int,
                    levels: int, xs, ys, mode: int = LEVEL_PAPER) -> np.ndarray:
    """(n, 3) uint8 R, G, B of the filtered pixels (xs[k], ys[k])."""
    src = np.ascontiguousarray(buf, dtype=np.uint8).reshape(-1)
    xs = np.ascontiguousarray(xs, dtype=np.uint32)
    ys = np.ascontiguousarray(ys, dtype=np.uint32)
    n = xs.size
    rgb = np.zeros((n, 3), dtype=np.uint8)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    rc = _load().orc_oilpaint_pixels(_u8(src), width, height, stride, bpp, radius, levels, mode,
                                     xs.ctypes.data_as(u32p), ys.ctypes.data_as(u32p), n,
                                     _u8(rgb))
    if rc != 0:
        raise ValueError(f"oracle rejected arguments (status {rc})")
    return rgb


def view_pixels(buf: np.ndarray, width: int, height: int, stride: int, bpp: int) -> np.ndarray:
    """(H, W, bpp) view of the pixel bytes of a strided buffer."""
    flat = np.asarray(buf).reshape(-1)
    return flat[: height * stride].reshape(height, stride)[:, : width * bpp].reshape(
        height, width, bpp)


__all__ = [
    "LEVEL_PAPER", "LEVEL_INTDIV3", "LITERAL", "level_map", "level_of_sum", "num_cpus", "oilpaint",
    "oilpaint_rows", "oilpaint_pixels", "oilpaint_numpy", "oilpaint_np", "view_pixels",
]
