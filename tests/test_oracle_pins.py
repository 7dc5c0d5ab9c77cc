"""The CPU oracles against their pins, against each other, and planted
mistakes against the pins (each must be caught)."""
import types

import numpy as np
import pytest

import oracle
from oracle import oilpaint_np as onp
from paper_1405_1020_gb300 import synth
from tests import pins


def c_oracle(buf, w, h, stride, bpp, r, L, mode, threads=0):
    out = np.full(np.asarray(buf).size, pins.OUT_FILL, dtype=np.uint8)
    return oracle.oilpaint(buf, w, h, stride, bpp, r, L, mode=mode, threads=threads, out=out)


def np_oracle(buf, w, h, stride, bpp, r, L, mode):
    out = np.full(np.asarray(buf).size, pins.OUT_FILL, dtype=np.uint8)
    return onp.oilpaint_buffer(buf, w, h, stride, bpp, r, L, mode, out=out)


ORACLES = {"c": c_oracle, "numpy": np_oracle}


@pytest.mark.parametrize("name", sorted(ORACLES))
@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda p: p.__name__)
def test_oracle_pin(name, pin):
    pin(ORACLES[name])


def test_single_thread_c_oracle_pins():
    for pin in pins.ALL_PINS:
        pin(lambda *a: c_oracle(*a, threads=1))


# ---- the two oracles agree byte for byte on random cases --------------------

def _cases():
    rng = np.random.default_rng(20)
    out = []
    for k in range(36):
        w = int(rng.integers(1, 60))
        h = int(rng.integers(1, 60))
        r = int(rng.choice([0, 1, 2, 3, 5, 8, 12, 20]))
        L = int(rng.choice([1, 2, 3, 16, 20, 32, 64, 255, 256]))
        bpp = int(rng.choice([3, 4]))
        pad = int(rng.choice([0, 1, 3, 16]))
        mode = int(rng.integers(0, 2))
        kind = int(rng.integers(0, 3))
        out.append((k, w, h, r, L, bpp, pad, mode, kind))
    return out


@pytest.mark.parametrize("k,w,h,r,L,bpp,pad,mode,kind", _cases())
def test_c_matches_numpy(k, w, h, r, L, bpp, pad, mode, kind):
    if kind == 0:
        img = synth.uniform_rgb(h, w, seed=100 + k)
    elif kind == 1:
        img = synth.blobs_rgb(h, w, seed=100 + k, nblobs=4, sigma_range=(2, 10))
    else:
        img = synth.camera_like(h, w, seed=100 + k, npoly=6, rad_range=(2, 30))
    buf, stride = synth.to_strided(img, bpp=bpp, stride=w * bpp + pad)
    a = c_oracle(buf, w, h, stride, bpp, r, L, mode)
    b = np_oracle(buf, w, h, stride, bpp, r, L, mode)
    assert np.array_equal(a, b)


def test_thread_count_invariance():
    img = synth.blobs_rgb(57, 61, seed=21, nblobs=5, sigma_range=(3, 15))
    buf, stride = synth.to_strided(img, bpp=3)
    ref = c_oracle(buf, 61, 57, stride, 3, 4, 20, 0, threads=1)
    for t in (2, 3, 7, 64):
        assert np.array_equal(c_oracle(buf, 61, 57, stride, 3, 4, 20, 0, threads=t), ref)


def test_rows_and_pixels_entry_points_match_whole_image():
    img = synth.camera_like(48, 70, seed=22, npoly=10, rad_range=(3, 40))
    buf, stride = synth.to_strided(img, bpp=4, stride=70 * 4 + 4)
    full = c_oracle(buf, 70, 48, stride, 4, 5, 20, 0)
    part = np.full(buf.size, pins.OUT_FILL, np.uint8)
    oracle.oilpaint_rows(buf, 70, 48, stride, 4, 5, 20, 10, 31, out=part)
    rows = slice(10 * stride, 31 * stride)
    assert np.array_equal(part[rows], full[rows])
    assert (part[: 10 * stride] == pins.OUT_FILL).all()
    rng = np.random.default_rng(23)
    xs = rng.integers(0, 70, 50)
    ys = rng.integers(0, 48, 50)
    rgb = oracle.oilpaint_pixels(buf, 70, 48, stride, 4, 5, 20, xs, ys)
    px = oracle.view_pixels(full, 70, 48, stride, 4)
    assert np.array_equal(rgb, px[ys, xs, :3])


def test_oracle_rejects_bad_arguments():
    buf = np.zeros(30, np.uint8)
    with pytest.raises(ValueError):
        oracle.oilpaint(buf, 5, 2, 14, 3, 1, 20)  # stride < width*bpp
    with pytest.raises(ValueError):
        oracle.oilpaint(buf, 5, 2, 15, 3, 1, 0)   # L = 0
    with pytest.raises(ValueError):
        oracle.oilpaint(buf, 5, 2, 15, 3, 1, 257)  # L > 256
    with pytest.raises(ValueError):
        oracle.oilpaint(buf, 5, 2, 15, 5, 1, 20)  # bpp 5


# ---- planted mistakes: every mutant must fail at least one pin ---------------

def _fails_some_pin(fn):
    failed = []
    for pin in pins.ALL_PINS:
        try:
            with np.errstate(all="ignore"):
                pin(fn)
        except (AssertionError, IndexError, ValueError, ZeroDivisionError, FloatingPointError):
            failed.append(pin.__name__)
    return failed


def _mut_no_clamp(rgb, levels, mode=0):
    s = rgb[..., 0].astype(np.int64) + rgb[..., 1] + rgb[..., 2]
    return ((s // 3) * levels) // 255 if mode == 1 else (s * levels) // 765


def _mut_divide_first(rgb, levels, mode=0):
    s = rgb[..., 0].astype(np.int64) + rgb[..., 1] + rgb[..., 2]
    return np.minimum(((s // 3) * levels) // 255, levels - 1)


def _mut_short_window(plane, r):
    h, w = plane.shape
    ii = np.zeros((h + 1, w + 1), dtype=np.int64)
    ii[1:, 1:] = plane.astype(np.int64).cumsum(0).cumsum(1)
    ys, xs = np.arange(h), np.arange(w)
    y0 = np.clip(ys - r, 0, h)[:, None]
    y1 = np.clip(ys + r, 0, h)[:, None]  # one row short
    x0 = np.clip(xs - r, 0, w)[None, :]
    x1 = np.clip(xs + r + 1, 0, w)[None, :]
    return ii[y1, x1] - ii[y0, x1] - ii[y1, x0] + ii[y0, x0]


def _np_with_last_argmax():
    proxy = types.SimpleNamespace(**{k: getattr(np, k) for k in dir(np) if not k.startswith("__")})
    proxy.argmax = lambda a, axis=None: a.shape[0] - 1 - np.argmax(a[::-1], axis=axis)
    return proxy


def _swap_channels(buf, w, h, stride, bpp, r, L, mode):
    out = np_oracle(buf, w, h, stride, bpp, r, L, mode)
    px = oracle.view_pixels(out, w, h, stride, bpp)
    px[..., [0, 2]] = px[..., [2, 0]]
    return out


def _black_outside(buf, w, h, stride, bpp, r, L, mode):
    """Counts out-of-image neighbours as black instead of skipping them."""
    px = oracle.view_pixels(buf, w, h, stride, bpp)
    big = np.zeros((h + 2 * r, w + 2 * r, bpp), np.uint8)
    big[r:r + h, r:r + w] = px
    res = onp.oilpaint_rgb(big, r, L, mode)[r:r + h, r:r + w]
    out = np.full(np.asarray(buf).size, pins.OUT_FILL, np.uint8)
    o = oracle.view_pixels(out, w, h, stride, bpp)
    o[..., :3] = res
    if bpp == 4:
        o[..., 3] = px[..., 3]
    return out


@pytest.mark.parametrize("mutant", ["no_clamp", "divide_first", "short_window", "tie_high",
                                    "swap_channels", "black_outside"])
def test_planted_mistake_is_caught(mutant, monkeypatch):
    fn = np_oracle
    if mutant == "no_clamp":
        monkeypatch.setattr(onp, "level_map", _mut_no_clamp)
    elif mutant == "divide_first":
        monkeypatch.setattr(onp, "level_map", _mut_divide_first)
    elif mutant == "short_window":
        monkeypatch.setattr(onp, "_box_sums", _mut_short_window)
    elif mutant == "tie_high":
        monkeypatch.setattr(onp, "np", _np_with_last_argmax())
    elif mutant == "swap_channels":
        fn = _swap_channels
    elif mutant == "black_outside":
        fn = _black_outside
    assert _fails_some_pin(fn), f"mutant {mutant} passed every pin"
