"""Pins of the oracle's literal mode: the section-4 listing as printed.

The listing visits only pixels at least `radius` from every edge, computes
the level without a clamp (pure white reaches level L), runs its argmax over
levels 0..L-1 only, writes nothing when all of those are empty, and writes
the three colour bytes.  Each pin below checks one of these facts against
something fixed independently of the oracle: a hand-derived example, closed
forms, the default mode on images where the readings coincide, and
convolution box sums.
"""
import json
import os

import numpy as np
import pytest
from scipy import signal

import oracle
from paper_1405_1020_gb300 import synth

from tests.pins import GOLDEN, OUT_FILL

LIT = oracle.LITERAL


def _lit(buf, w, h, stride, bpp, r, L, mode=LIT):
    out = np.full(np.asarray(buf).size, OUT_FILL, np.uint8)
    return oracle.oilpaint(buf, w, h, stride, bpp, r, L, mode=mode, out=out)


def _pix(out, w, h, stride, bpp):
    return oracle.view_pixels(out, w, h, stride, bpp)


def _interior(r, w, h):
    m = np.zeros((h, w), bool)
    if w > 2 * r and h > 2 * r:
        m[r:h - r, r:w - r] = True
    return m


def pin_literal_worked_example(fn):
    with open(os.path.join(GOLDEN, "literal_white_exclusion.json")) as f:
        g = json.load(f)
    img = np.array(g["pixels_rgb_rows"], np.uint8)
    h, w = img.shape[:2]
    buf = img.reshape(-1).copy()
    px = _pix(fn(buf, w, h, w * 3, 3, g["radius"], g["levels"]), w, h, w * 3, 3)
    c = g["check"]
    assert px[c["y"], c["x"]].tolist() == c["literal_rgb"]
    border = ~_interior(g["radius"], w, h)
    assert (px[border] == OUT_FILL).all(), "the listing does not visit border pixels"


def pin_literal_all_white_writes_nothing(fn):
    img = np.full((9, 12, 3), 255, np.uint8)
    for bpp, r, L in ((3, 1, 20), (4, 2, 254), (3, 0, 1)):
        buf, stride = synth.to_strided(img, bpp=bpp, stride=12 * bpp + 4)
        out = fn(buf, 12, 9, stride, bpp, r, L)
        assert (_pix(out, 12, 9, stride, bpp) == OUT_FILL).all(), (bpp, r, L)


def pin_literal_equals_default_inside_without_white(fn):
    """Without a pure-white pixel no level reaches L, and interior windows
    are never clipped, so the literal interior must equal the default
    filter there; the border, row padding and alpha stay untouched."""
    img = synth.camera_like(41, 57, seed=5, npoly=15, rad_range=(2, 30))
    img[img.sum(axis=2) == 765] = (254, 255, 255)
    for bpp, r, L, mode in ((3, 2, 20, 0), (4, 5, 7, 1), (3, 0, 254, 0), (4, 9, 64, 0)):
        buf, stride = synth.to_strided(img, bpp=bpp, stride=57 * bpp + 3)
        got = fn(buf, 57, 41, stride, bpp, r, L, LIT | mode)
        want = oracle.oilpaint(buf, 57, 41, stride, bpp, r, L, mode=mode)
        g, e = _pix(got, 57, 41, stride, bpp), _pix(want, 57, 41, stride, bpp)
        inside = _interior(r, 57, 41)
        assert np.array_equal(g[inside][:, :3], e[inside][:, :3]), (bpp, r, L, mode)
        assert (g[~inside] == OUT_FILL).all()
        if bpp == 4:
            assert (g[..., 3] == OUT_FILL).all(), "the listing writes three bytes"
        pad = np.asarray(got).reshape(-1)[: 41 * stride].reshape(41, stride)[:, 57 * bpp:]
        assert (pad == OUT_FILL).all()


def pin_literal_one_level_is_mean_of_non_white(fn):
    """L = 1: every non-white pixel is level 0 and white is level 1 (never
    read), so each interior output is the truncated mean of the window's
    non-white pixels, or unwritten if there are none."""
    rng = np.random.default_rng(9)
    img = rng.integers(0, 256, (30, 26, 3)).astype(np.uint8)
    white = rng.random((30, 26)) < 0.4
    img[white] = 255
    r = 2
    buf = img.reshape(-1).copy()
    px = _pix(fn(buf, 26, 30, 78, 3, r, 1), 26, 30, 78, 3)
    k = np.ones((2 * r + 1, 2 * r + 1), np.int64)
    keep = (~white).astype(np.int64)
    cnt = np.rint(signal.convolve2d(keep, k, mode="same")).astype(np.int64)
    inside = _interior(r, 26, 30)
    for c in range(3):
        s = np.rint(signal.convolve2d(img[..., c].astype(np.int64) * keep, k, mode="same"))
        s = s.astype(np.int64)
        ok = inside & (cnt > 0)
        assert np.array_equal(px[..., c][ok], s[ok] // cnt[ok]), c
    assert (px[inside & (cnt == 0)] == OUT_FILL).all()
    assert (px[~inside] == OUT_FILL).all()


def pin_literal_small_images_untouched(fn):
    img = synth.uniform_rgb(6, 9, seed=2)
    for r in (3, 4, 5):  # w = 9 > 2r only for r <= 4, h = 6 > 2r only for r <= 2
        buf = img.reshape(-1).copy()
        px = _pix(fn(buf, 9, 6, 27, 3, r, 20), 9, 6, 27, 3)
        assert (px == OUT_FILL).all(), r


PINS = [pin_literal_worked_example, pin_literal_all_white_writes_nothing,
        pin_literal_equals_default_inside_without_white, pin_literal_one_level_is_mean_of_non_white,
        pin_literal_small_images_untouched]


@pytest.mark.parametrize("pin", PINS, ids=lambda p: p.__name__)
def test_literal_pin(pin):
    pin(_lit)


def test_default_mode_differs_on_the_worked_example():
    with open(os.path.join(GOLDEN, "literal_white_exclusion.json")) as f:
        g = json.load(f)
    img = np.array(g["pixels_rgb_rows"], np.uint8)
    out = oracle.oilpaint(img.reshape(-1).copy(), 3, 3, 9, 3, 1, 20)
    assert _pix(out, 3, 3, 9, 3)[1, 1].tolist() == g["check"]["default_rgb"]


def test_literal_argument_limits():
    buf = np.zeros(4 * 4 * 3, np.uint8)
    with pytest.raises(ValueError):
        oracle.oilpaint(buf, 4, 4, 12, 3, 1, 255, mode=LIT)  # level L must fit 255 entries
    with pytest.raises(ValueError):
        oracle.oilpaint_pixels(buf, 4, 4, 12, 3, 1, 20, [0], [0], mode=LIT)
    with pytest.raises(ValueError):
        oracle.oilpaint_numpy(buf, 4, 4, 12, 3, 1, 20, mode=LIT)


def _mut_default_mode(buf, w, h, stride, bpp, r, L, mode=LIT):
    return _lit(buf, w, h, stride, bpp, r, L, mode & ~LIT)


def _mut_writes_border(buf, w, h, stride, bpp, r, L, mode=LIT):
    out = _lit(buf, w, h, stride, bpp, r, L, mode)
    full = oracle.oilpaint(buf, w, h, stride, bpp, r, L, mode=mode & ~LIT)
    pb = _pix(out, w, h, stride, bpp)
    border = ~_interior(r, w, h)
    pb[border] = _pix(full, w, h, stride, bpp)[border]
    return out


@pytest.mark.parametrize("mutant", [_mut_default_mode, _mut_writes_border],
                         ids=lambda m: m.__name__)
def test_planted_literal_mistake_is_caught(mutant):
    failed = 0
    for pin in PINS:
        try:
            pin(mutant)
        except AssertionError:
            failed += 1
    assert failed, f"{mutant.__name__} passes every literal pin"
