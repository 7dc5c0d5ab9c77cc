"""Seeded synthetic images and workloads.

This module holds none of the filter's arithmetic: it only makes inputs.  The
paper measured unnamed JPEG camera photos from VGA to WQXGA (section 4,
Experimental Results); those photos are not available, so seeded synthetic
images with the shapes and the kind of structure of camera photos stand in for
them:

* ``uniform_rgb``   -- i.i.d. uniform bytes (the worst case for histogram
  coherence: every window is close to flat across levels);
* ``blobs_rgb``     -- a piecewise-smooth field: grey 128 plus 64 Gaussian
  colour blobs (sigma 40..200 px, per-channel amplitude -160..160) plus
  per-pixel Gaussian noise;
* ``camera_like``   -- smooth gradients (three random linear ramps per channel
  and a low-frequency cosine) overpainted by 200 sharp-edged random polygons
  (3-8 vertices, radius 20..600 px, uniform random colours, even-odd fill)
  plus Gaussian noise;
* ``to_strided``    -- lays an (H, W, 3) image out as RGB or RGBA rows with a
  row pitch and a canary pattern in the row padding;
* ``batch_specs`` / ``poisson_requests`` -- the mixed batch and the request
  stream of the batched and served workloads.

All randomness comes from ``numpy.random.default_rng(seed)``; values are
rounded with ``np.rint`` and clipped to 0..255.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CANARY = 0xA5


def uniform_rgb(height: int, width: int, seed: int = 0) -> np.ndarray:
    """i.i.d. uniform 0..255 per channel, shape (H, W, 3) uint8."""
    return np.random.default_rng(seed).integers(0, 256, (height, width, 3), dtype=np.uint8)


def _finish(f: np.ndarray) -> np.ndarray:
    return np.clip(np.rint(f), 0, 255).astype(np.uint8)


def blobs_rgb(height: int, width: int, seed: int = 1, nblobs: int = 64,
              sigma_range=(40.0, 200.0), amp: float = 160.0, noise: float = 8.0) -> np.ndarray:
    """Grey 128 + `nblobs` Gaussian colour blobs + N(0, noise^2) per pixel."""
    rng = np.random.default_rng(seed)
    f = np.full((height, width, 3), 128.0, dtype=np.float64)
    ys = np.arange(height, dtype=np.float64)
    xs = np.arange(width, dtype=np.float64)
    for _ in range(nblobs):
        cy = rng.uniform(0, height)
        cx = rng.uniform(0, width)
        sig = rng.uniform(*sigma_range)
        a = rng.uniform(-amp, amp, size=3)
        y0, y1 = max(0, int(cy - 4 * sig)), min(height, int(cy + 4 * sig) + 1)
        x0, x1 = max(0, int(cx - 4 * sig)), min(width, int(cx + 4 * sig) + 1)
        if y0 >= y1 or x0 >= x1:
            continue
        gy = np.exp(-0.5 * ((ys[y0:y1] - cy) / sig) ** 2)
        gx = np.exp(-0.5 * ((xs[x0:x1] - cx) / sig) ** 2)
        g = gy[:, None] * gx[None, :]
        f[y0:y1, x0:x1, :] += g[:, :, None] * a[None, None, :]
    f += rng.normal(0.0, noise, size=f.shape)
    return _finish(f)


def _fill_polygon(img: np.ndarray, vx: np.ndarray, vy: np.ndarray, colour: np.ndarray) -> None:
    """Even-odd scanline fill of one polygon, sampling at pixel centres."""
    h, w = img.shape[:2]
    ymin = max(0, int(math.floor(vy.min())))
    ymax = min(h - 1, int(math.ceil(vy.max())))
    xmin = max(0, int(math.floor(vx.min())))
    xmax = min(w - 1, int(math.ceil(vx.max())))
    if ymin > ymax or xmin > xmax:
        return
    yc = np.arange(ymin, ymax + 1, dtype=np.float64) + 0.5
    x1, y1 = vx, vy
    x2, y2 = np.roll(vx, -1), np.roll(vy, -1)
    lo = np.minimum(y1, y2)[None, :]
    hi = np.maximum(y1, y2)[None, :]
    crosses = (yc[:, None] >= lo) & (yc[:, None] < hi)
    dy = np.where(y2 != y1, y2 - y1, 1.0)
    xi = x1[None, :] + (yc[:, None] - y1[None, :]) * ((x2 - x1) / dy)[None, :]
    # first pixel column whose centre lies right of the crossing
    col = np.floor(xi - 0.5).astype(np.int64) + 1 - xmin
    bw = xmax - xmin + 1
    col = np.clip(col, 0, bw)
    rows = np.broadcast_to(np.arange(yc.size)[:, None], col.shape)
    flat = rows[crosses] * (bw + 1) + col[crosses]
    diff = np.bincount(flat, minlength=yc.size * (bw + 1)).astype(np.uint8)
    diff = diff.reshape(yc.size, bw + 1)[:, :bw]
    inside = (np.bitwise_xor.accumulate(diff & 1, axis=1)).astype(bool)
    region = img[ymin:ymax + 1, xmin:xmax + 1]
    region[inside] = colour


def camera_like(height: int, width: int, seed: int = 2, npoly: int = 200, noise: float = 6.0,
                rad_range=(20.0, 600.0)) -> np.ndarray:
    """Smooth gradients + `npoly` sharp-edged polygons + N(0, noise^2)."""
    rng = np.random.default_rng(seed)
    yy = (np.arange(height, dtype=np.float64) / max(1, height))[:, None]
    xx = (np.arange(width, dtype=np.float64) / max(1, width))[None, :]
    f = np.empty((height, width, 3), dtype=np.float64)
    for c in range(3):
        ch = np.full((height, width), rng.uniform(60, 200))
        for _ in range(3):
            th = rng.uniform(0, 2 * math.pi)
            ch = ch + rng.uniform(-60, 60) * (math.cos(th) * xx + math.sin(th) * yy)
        fx, fy = rng.uniform(0.5, 2.0, size=2)
        ch = ch + rng.uniform(10, 40) * np.cos(2 * math.pi * (fx * xx + fy * yy)
                                               + rng.uniform(0, 2 * math.pi))
        f[..., c] = ch
    img = _finish(f)
    for _ in range(npoly):
        nv = int(rng.integers(3, 9))
        cx = rng.uniform(0, width)
        cy = rng.uniform(0, height)
        rad = rng.uniform(*rad_range)
        ang = rng.uniform(0, 2 * math.pi, size=nv)
        rr = rad * rng.uniform(0.4, 1.0, size=nv)
        colour = rng.integers(0, 256, size=3, dtype=np.uint8)
        _fill_polygon(img, cx + rr * np.cos(ang), cy + rr * np.sin(ang), colour)
    out = img.astype(np.float64) + rng.normal(0.0, noise, size=img.shape)
    return _finish(out)


def to_strided(img: np.ndarray, bpp: int = 3, stride: int | None = None, alpha: int = 255,
               pad_value: int = CANARY) -> tuple[np.ndarray, int]:
    """Lay an (H, W, 3) image out in rows of `stride` bytes, `bpp` bytes per
    pixel (alpha = `alpha` when bpp == 4), padding bytes set to `pad_value`.
    Returns (flat uint8 buffer of H*stride bytes, stride)."""
    h, w = img.shape[:2]
    if bpp not in (3, 4):
        raise ValueError("bpp must be 3 or 4")
    if stride is None:
        stride = w * bpp
    if stride < w * bpp:
        raise ValueError("stride smaller than a row")
    buf = np.full((h, stride), pad_value, dtype=np.uint8)
    px = buf[:, : w * bpp].reshape(h, w, bpp)
    px[..., :3] = img[..., :3]
    if bpp == 4:
        px[..., 3] = alpha
    return buf.reshape(-1), stride


@dataclass(frozen=True)
class ImageSpec:
    """One image of a mixed batch."""
    width: int
    height: int
    radius: int
    levels: int
    seed: int


def log_uniform_size(rng: np.random.Generator, pmin: float, pmax: float) -> tuple[int, int]:
    """(w, h) with w*h log-uniform in [pmin, pmax] and aspect 4:3 or 16:9."""
    p = math.exp(rng.uniform(math.log(pmin), math.log(pmax)))
    a = 4.0 / 3.0 if rng.random() < 0.5 else 16.0 / 9.0
    w = max(1, int(round(math.sqrt(p * a))))
    h = max(1, int(round(p / w)))
    return w, h


def batch_specs(n: int = 64, seed: int = 3, pmin: float = 320 * 240, pmax: float = 4000 * 3000,
                radii=(2, 4, 8, 12, 20), levels=(16, 20, 32)) -> list[ImageSpec]:
    """The mixed batch: sizes log-uniform in [pmin, pmax] pixels, radius and
    level count uniform over the given sets."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        w, h = log_uniform_size(rng, pmin, pmax)
        r = int(rng.choice(radii))
        L = int(rng.choice(levels))
        out.append(ImageSpec(w, h, r, L, seed * 1000 + i))
    return out


@dataclass(frozen=True)
class Request:
    """One served request: arrival time (s from start), size, radius, levels,
    and the crop origin inside the device-resident image pool."""
    t_arrival: float
    width: int
    height: int
    radius: int
    levels: int
    pool_index: int
    x0: int
    y0: int


def poisson_requests(rate_per_s: float, duration_s: float, seed: int = 4, pmin: float = 0.1e6,
                     pmax: float = 24e6, rmin: int = 1, rmax: int = 20, levels: int = 20,
                     pool_shapes=((4000, 6000),)) -> list[Request]:
    """Poisson arrivals at `rate_per_s` for `duration_s` seconds; sizes
    log-uniform in [pmin, pmax] pixels (aspect 4:3 or 16:9, either
    orientation that fits the pool), radius uniform in rmin..rmax."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t >= duration_s:
            break
        w, h = log_uniform_size(rng, pmin, pmax)
        k = int(rng.integers(0, len(pool_shapes)))
        ph, pw = pool_shapes[k]
        if w > pw or h > ph:
            w, h = h, w
        w, h = min(w, pw), min(h, ph)
        r = int(rng.integers(rmin, rmax + 1))
        x0 = int(rng.integers(0, pw - w + 1))
        y0 = int(rng.integers(0, ph - h + 1))
        reqs.append(Request(t, w, h, r, levels, k, x0, y0))
    return reqs
