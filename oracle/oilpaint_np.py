"""Second, independent CPU oracle in NumPy -- TEST INFRASTRUCTURE ONLY.

It computes the same function as ``oilpaint_ref.c`` (the histogram oil-paint
filter of section 4 of Mukherjee, arXiv 1405.1020) by a different algorithm:

* the level map of the whole image first (section 4's intensity level,
  floor((R+G+B) * L / 765), clamped to L-1; or the divide-by-3-first mode);
* for every level l, integral images (2-D prefix sums) of the indicator
  [level == l] and of R, G, B masked by it, so that the count and the three
  sums of level l over any clipped window are four table reads;
* the argmax over levels with ``np.argmax``, which returns the first maximum,
  i.e. the lowest level on a tie (section 4's most frequent intensity with the
  lowest-level convention);
* truncating integer division of the winning sums by the winning count.

Windows are clipped at the image border (out-of-image neighbours skipped).
It shares no code with the C oracle or the CUDA path.  Memory is
O(L * H * W), so it is meant for small and medium images.
"""
from __future__ import annotations

import numpy as np

LEVEL_PAPER = 0
LEVEL_INTDIV3 = 1


def level_map(rgb: np.ndarray, levels: int, mode: int = LEVEL_PAPER) -> np.ndarray:
    """Per-pixel intensity level (section 4), clamped to levels-1."""
    s = rgb[..., 0].astype(np.int64) + rgb[..., 1] + rgb[..., 2]
    if mode == LEVEL_INTDIV3:
        lv = ((s // 3) * levels) // 255
    else:
        lv = (s * levels) // 765
    return np.minimum(lv, levels - 1)


def _box_sums(plane: np.ndarray, r: int) -> np.ndarray:
    """Sum of `plane` over the (2r+1)^2 window clipped to the image."""
    h, w = plane.shape
    ii = np.zeros((h + 1, w + 1), dtype=np.int64)
    ii[1:, 1:] = plane.astype(np.int64).cumsum(0).cumsum(1)
    ys = np.arange(h)
    xs = np.arange(w)
    y0 = np.clip(ys - r, 0, h)[:, None]
    y1 = np.clip(ys + r + 1, 0, h)[:, None]
    x0 = np.clip(xs - r, 0, w)[None, :]
    x1 = np.clip(xs + r + 1, 0, w)[None, :]
    return ii[y1, x1] - ii[y0, x1] - ii[y1, x0] + ii[y0, x0]


def oilpaint_rgb(rgb: np.ndarray, radius: int, levels: int, mode: int = LEVEL_PAPER) -> np.ndarray:
    """Filter an (H, W, >=3) uint8 array; returns the (H, W, 3) uint8 result."""
    if rgb.ndim != 3 or rgb.shape[2] < 3:
        raise ValueError("expected an (H, W, C>=3) array")
    h, w = rgb.shape[:2]
    lv = level_map(rgb, levels, mode)
    chans = [rgb[..., c].astype(np.int64) for c in range(3)]
    counts = np.empty((levels, h, w), dtype=np.int64)
    sums = np.empty((levels, 3, h, w), dtype=np.int64)
    for l in range(levels):
        ind = lv == l
        counts[l] = _box_sums(ind, radius)
        for c in range(3):
            sums[l, c] = _box_sums(np.where(ind, chans[c], 0), radius)
    best = np.argmax(counts, axis=0)  # first maximum -> lowest level
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    cnt = counts[best, yy, xx]
    out = np.empty((h, w, 3), dtype=np.uint8)
    for c in range(3):
        out[..., c] = (sums[best, c, yy, xx] // cnt).astype(np.uint8)
    return out


def oilpaint_buffer(buf: np.ndarray, width: int, height: int, stride: int, bpp: int,
                    radius: int, levels: int, mode: int = LEVEL_PAPER,
                    out: np.ndarray | None = None) -> np.ndarray:
    """Same filter on a strided byte buffer of height*stride bytes.

    Only pixel bytes are written; with bpp == 4 the alpha byte is copied from
    the input.  `out` (same size as `buf`) keeps its row padding.
    """
    if mode not in (LEVEL_PAPER, LEVEL_INTDIV3):
        raise ValueError("the NumPy oracle implements the two level modes only")
    flat = np.ascontiguousarray(buf).reshape(-1)
    if flat.size < height * stride:
        raise ValueError("buffer too small")
    rows = flat[: height * stride].reshape(height, stride)
    img = rows[:, : width * bpp].reshape(height, width, bpp)
    res = oilpaint_rgb(img, radius, levels, mode)
    if out is None:
        out = np.zeros_like(flat)
    o = out.reshape(-1)
    orows = o[: height * stride].reshape(height, stride)
    opix = orows[:, : width * bpp].reshape(height, width, bpp)
    opix[..., :3] = res
    if bpp == 4:
        opix[..., 3] = img[..., 3]
    return out
