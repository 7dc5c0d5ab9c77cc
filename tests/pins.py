"""Pins for a CPU oracle of the section-4 oil-paint filter.

Each pin takes an oracle callable
    oracle(buf, width, height, stride, bpp, radius, levels, mode) -> out buffer
and raises AssertionError if the oracle disagrees with something fixed
independently of it: the paper's described example, closed forms (identity,
box mean), textbook library routines (scipy convolution, min/max filters),
symmetries of the definition, or brute-force counting by another method.
"""
from __future__ import annotations

import json
import os

import numpy as np
from scipy import ndimage, signal

from paper_1405_1020_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PAPER, INTDIV3 = 0, 1
# Oracle callables start from an output buffer filled with this byte, so that
# bytes they do not write are recognisable.
OUT_FILL = 0x5A


def _run(oracle, img, radius, levels, mode=PAPER, bpp=3, pad=0):
    h, w = img.shape[:2]
    buf, stride = synth.to_strided(img, bpp=bpp, stride=w * bpp + pad)
    out = oracle(buf, w, h, stride, bpp, radius, levels, mode)
    out = np.asarray(out).reshape(-1)
    px = out[: h * stride].reshape(h, stride)[:, : w * bpp].reshape(h, w, bpp)
    return px, out, stride


def _window_counts(mask: np.ndarray, r: int) -> np.ndarray:
    k = np.ones((2 * r + 1, 2 * r + 1), dtype=np.int64)
    return np.rint(signal.convolve2d(mask.astype(np.int64), k, mode="same")).astype(np.int64)


def pin_golden_sec4(oracle):
    """Section 4's described radius-1 example (fixture values, see the file)."""
    with open(os.path.join(GOLDEN, "worked_example_sec4.json")) as f:
        g = json.load(f)
    img = np.array(g["pixels_rgb_rows"], dtype=np.uint8)
    px, _, _ = _run(oracle, img, g["radius"], g["levels"])
    c = g["check"]
    got = px[c["y"], c["x"], :3].tolist()
    assert got == c["expected_rgb"], f"section-4 example: got {got}, want {c['expected_rgb']}"


def pin_identity_r0(oracle):
    """r = 0: the window is the pixel itself, so the output is the input."""
    img = synth.uniform_rgb(23, 37, seed=11)
    for bpp, pad in ((3, 0), (3, 5), (4, 8)):
        px, out, stride = _run(oracle, img, 0, 20, bpp=bpp, pad=pad)
        assert np.array_equal(px[..., :3], img), "r=0 must be the identity"
        if bpp == 4:
            assert (px[..., 3] == 255).all(), "alpha must be copied"


def pin_constant_identity(oracle):
    """A constant image is its own oil paint, whatever r and L (white too)."""
    for colour in ((255, 255, 255), (0, 0, 0), (17, 200, 3), (128, 128, 127)):
        img = np.empty((9, 13, 3), dtype=np.uint8)
        img[:] = colour
        for L in (1, 7, 20, 256):
            for r in (1, 3, 6):
                px, _, _ = _run(oracle, img, r, L)
                assert (px[..., :3] == np.array(colour, np.uint8)).all(), (
                    f"constant {colour} L={L} r={r} not preserved")


def pin_box_mean_L1(oracle):
    """L = 1 puts every pixel in one level: the output is the truncated mean
    over the clipped window (sums and counts by scipy convolution)."""
    cases = [(synth.uniform_rgb(29, 41, seed=12), r) for r in (1, 2, 5)]
    cases.append((synth.uniform_rgb(4, 5, seed=13), 5))  # smaller than the window
    for img, r in cases:
        px, _, _ = _run(oracle, img, r, 1)
        cnt = _window_counts(np.ones(img.shape[:2]), r)
        for c in range(3):
            s = _window_counts(img[..., c], r)
            want = (s // cnt).astype(np.uint8)
            assert np.array_equal(px[..., c], want), f"L=1 box mean r={r} channel {c}"


def pin_two_colour(oracle):
    """Two colours in different levels: every pixel takes the colour with more
    window members, the lower level on a tie; two colours in one level: the
    truncated mean of the window's members."""
    rng = np.random.default_rng(14)
    A = np.array([10, 20, 30], np.uint8)     # R+G+B =  60 -> level  1 of 20
    B = np.array([200, 210, 220], np.uint8)  # R+G+B = 630 -> level 16 of 20
    mask = rng.random((31, 27)) < 0.5
    img = np.where(mask[..., None], B, A).astype(np.uint8)
    for r in (1, 2, 4):
        px, _, _ = _run(oracle, img, r, 20)
        nb = _window_counts(mask, r)
        na = _window_counts(~mask, r)
        want = np.where((nb > na)[..., None], B, A)
        assert np.array_equal(px[..., :3], want), f"two-colour majority r={r}"
    # an exact tie: both pixels of a 2x1 image see one A and one B
    px, _, _ = _run(oracle, np.stack([A, B])[None], 1, 20)
    assert (px[..., :3] == A).all(), "tie must go to the lower level"
    # same level: R+G+B = 180 and 190 are both level 4 of 20
    C = np.array([100, 50, 30], np.uint8)
    D = np.array([40, 90, 60], np.uint8)
    img = np.where(mask[..., None], D, C).astype(np.uint8)
    r = 2
    px, _, _ = _run(oracle, img, r, 20)
    nd = _window_counts(mask, r)
    nc = _window_counts(~mask, r)
    for c in range(3):
        want = (nd * int(D[c]) + nc * int(C[c])) // (nd + nc)
        assert np.array_equal(px[..., c], want.astype(np.uint8)), "same-level mean"


def pin_window_range(oracle):
    """Every output channel lies within that channel's range over the window."""
    img = synth.blobs_rgb(40, 52, seed=15, nblobs=6, sigma_range=(3, 12))
    for r, L in ((3, 16), (2, 256), (5, 3)):
        px, _, _ = _run(oracle, img, r, L)
        for c in range(3):
            lo = ndimage.minimum_filter(img[..., c], size=2 * r + 1, mode="nearest")
            hi = ndimage.maximum_filter(img[..., c], size=2 * r + 1, mode="nearest")
            assert (px[..., c] >= lo).all() and (px[..., c] <= hi).all(), "outside window range"


def pin_equivariance(oracle):
    """Flips and transposition commute with the filter (square window, ties
    broken by level not by position); permuting channels permutes the output
    (the level depends only on R+G+B)."""
    img = synth.uniform_rgb(19, 26, seed=16)
    r, L = 2, 12
    base, _, _ = _run(oracle, img, r, L)
    base = base[..., :3]
    for f in (lambda a: a[::-1], lambda a: a[:, ::-1], lambda a: a.transpose(1, 0, 2)):
        px, _, _ = _run(oracle, np.ascontiguousarray(f(img)), r, L)
        assert np.array_equal(px[..., :3], f(base)), "flip/transpose equivariance"
    perm = [2, 0, 1]
    px, _, _ = _run(oracle, np.ascontiguousarray(img[..., perm]), r, L)
    assert np.array_equal(px[..., :3], base[..., perm]), "channel permutation"


def pin_translation(oracle):
    """Pixels whose window lies inside an image keep their value when the
    image is embedded in a larger canvas."""
    r, L = 3, 20
    small = synth.uniform_rgb(20, 17, seed=17)
    canvas = synth.uniform_rgb(45, 50, seed=18)
    oy, ox = 13, 11
    canvas[oy:oy + 20, ox:ox + 17] = small
    a, _, _ = _run(oracle, small, r, L)
    b, _, _ = _run(oracle, canvas, r, L)
    inner_a = a[r:20 - r, r:17 - r, :3]
    inner_b = b[oy + r:oy + 20 - r, ox + r:ox + 17 - r, :3]
    assert np.array_equal(inner_a, inner_b), "translation invariance of interior pixels"


def pin_level_modes(oracle):
    """R+G+B = 77 is level 2 of 20 by section 4's formula and level 1 when
    dividing by 3 first; R+G+B = 80 is level 2 both ways.  Radius 1 on the
    row [77, 80, 80]: the clipped windows are {0,1}, {0,1,2}, {1,2}.  With the
    paper's levels all pixels share one level (window means); dividing first,
    pixel 0 sees a one-one tie (lower level: the 77 colour) and the others a
    majority of the 80 colour."""
    A = np.array([25, 26, 26], np.uint8)  # 77
    B = np.array([27, 27, 26], np.uint8)  # 80
    img = np.stack([A, B, B])[None]
    a, b = A.astype(int), B.astype(int)
    px, _, _ = _run(oracle, img, 1, 20, mode=PAPER)
    want = np.stack([(a + b) // 2, (a + 2 * b) // 3, b])
    assert (px[0, :, :3] == want).all(), "paper level mode: one shared level"
    px, _, _ = _run(oracle, img, 1, 20, mode=INTDIV3)
    want = np.stack([a, b, b])
    assert (px[0, :, :3] == want).all(), "divide-by-3-first mode: tie then majority"


def pin_padding_untouched(oracle):
    """Row padding keeps its bytes."""
    img = synth.uniform_rgb(11, 7, seed=19)
    for bpp in (3, 4):
        h, w = img.shape[:2]
        buf, stride = synth.to_strided(img, bpp=bpp, stride=w * bpp + 9)
        out = np.asarray(oracle(buf, w, h, stride, bpp, 2, 20, PAPER)).reshape(-1)
        rows = out[: h * stride].reshape(h, stride)
        assert (rows[:, w * bpp:] == OUT_FILL).all(), "row padding was written"


ALL_PINS = [pin_golden_sec4, pin_identity_r0, pin_constant_identity, pin_box_mean_L1,
            pin_two_colour, pin_window_range, pin_equivariance, pin_translation,
            pin_level_modes, pin_padding_untouched]
