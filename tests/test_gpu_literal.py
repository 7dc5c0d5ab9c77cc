"""Literal mode (OP_LITERAL) of the CUDA path against the oracle's literal
mode, byte for byte over the whole buffer: interior pixels, the untouched
border, alpha and row padding, and the pixels left unwritten because their
window holds only pure white."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from paper_1405_1020_gb300 import binding as B
from paper_1405_1020_gb300 import synth
from paper_1405_1020_gb300.filter import Batch, OilPaint
from tests.pins import OUT_FILL
from tests.test_gpu_parity import assert_same, cpu_filter, gpu_filter

pytestmark = pytest.mark.gpu
LIT = B.OP_LITERAL


@pytest.fixture(scope="module", autouse=True)
def _lib():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def whitened(h, w, seed, frac=0.3, blob=True):
    """Camera-like image with pure-white pixels: scattered ones and, with
    `blob`, a white rectangle larger than small windows."""
    img = synth.camera_like(h, w, seed=seed, npoly=12, rad_range=(2, 40))
    rng = np.random.default_rng(seed)
    img[rng.random((h, w)) < frac] = 255
    if blob and h > 8 and w > 8:
        img[h // 4: h // 4 + max(3, h // 3), w // 5: w // 5 + max(3, w // 3)] = 255
    return img


def check(img, r, L, bpp=3, pad=0, mode=0, config=None):
    h, w = img.shape[:2]
    buf, stride = synth.to_strided(img, bpp=bpp, stride=w * bpp + pad)
    got = gpu_filter(buf, w, h, stride, bpp, r, L, mode | LIT, config)
    want = cpu_filter(buf, w, h, stride, bpp, r, L, mode | LIT)
    assert_same(got, want, w, h, stride, bpp, f"literal {w}x{h} r={r} L={L} bpp={bpp} {config}")


@pytest.mark.parametrize("r,L", [(0, 20), (1, 1), (2, 20), (5, 7), (15, 20), (15, 32), (16, 20),
                                 (20, 32), (9, 64), (15, 254), (44, 20), (3, 2)])
@pytest.mark.parametrize("cpt,path", [(1, 0), (2, 0), (4, 0), (1, 1), (2, 1)])
def test_literal_matches_oracle(r, L, cpt, path):
    img = whitened(120, 211, seed=r * 31 + L)
    for bpp, pad, nt in ((3, 1, 32), (4, 8, 64)):
        cfg = {"tile_w": nt * cpt, "cols_per_thread": cpt, "chunk_rows": 4, "path": path}
        try:
            check(img, r, L, bpp, pad, 0, cfg)
        except B.OilPaintError as e:
            # K columns need L <= 32; some boxes / histograms do not fit
            assert e.status == B.OP_E_UNSUPPORTED, e


@pytest.mark.parametrize("w,h,r", [(5, 5, 2), (4, 9, 2), (9, 4, 2), (7, 7, 3), (3, 3, 1), (1, 1, 0),
                                   (30, 2, 1)])
def test_literal_small_images(w, h, r):
    """Images with no pixel r from every edge (nothing written) or only a
    few; the output must equal the oracle's (the fill byte where unwritten)."""
    check(whitened(h, w, seed=w * h + r, frac=0.2, blob=False), r, 20)
    check(whitened(h, w, seed=w * h + r + 1, frac=0.2, blob=False), r, 20, bpp=4, pad=4)


def test_literal_all_white_writes_nothing():
    img = np.full((64, 96, 3), 255, np.uint8)
    for r, L in ((2, 20), (17, 32), (3, 200)):
        buf, stride = synth.to_strided(img, bpp=4, stride=96 * 4)
        got = gpu_filter(buf, 96, 64, stride, 4, r, L, LIT)
        assert (got == OUT_FILL).all()


def test_literal_intdiv3_and_batch_mixed_with_default():
    """A batch mixing literal and default images (both level modes) equals
    the solo runs and the oracle."""
    rng = np.random.default_rng(5)
    images = []
    for k in range(10):
        h, w = int(rng.integers(20, 300)), int(rng.integers(20, 400))
        r = int(rng.choice([1, 4, 15, 20]))
        L = int(rng.choice([16, 20, 32]))
        mode = int(rng.integers(0, 2)) | (LIT if k % 2 else 0)
        img = whitened(h, w, seed=100 + k)
        buf, stride = synth.to_strided(img, bpp=3, stride=w * 3 + 2)
        src = torch.from_numpy(buf).cuda()
        images.append({"w": w, "h": h, "r": r, "L": L, "mode": mode, "stride": stride,
                       "buf": buf, "src": src, "dst": torch.full_like(src, OUT_FILL)})
    pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
    for cfg in (None, {"tile_w": 64, "chunk_rows": 2, "prefetch": 1, "cols_per_thread": 2}):
        b = Batch(16, pix + 64, 20, 32, config=cfg)
        for im in images:
            im["dst"].fill_(OUT_FILL)
        torch.cuda.synchronize()
        b.set([(im["src"], im["dst"], im["w"], im["h"], im["stride"], 3, im["r"], im["L"],
                im["mode"]) for im in images])
        b.run()
        assert b.sync_status() == B.OP_OK
        for im in images:
            want = cpu_filter(im["buf"], im["w"], im["h"], im["stride"], 3, im["r"], im["L"],
                              im["mode"])
            assert_same(im["dst"].cpu().numpy(), want, im["w"], im["h"], im["stride"], 3,
                        f"batch image mode={im['mode']} r={im['r']} L={im['L']}")
        b.close()


def test_literal_noalloc_and_limits():
    img = whitened(90, 130, seed=3)
    buf, stride = synth.to_strided(img, bpp=4, stride=130 * 4)
    src = torch.from_numpy(buf).cuda()
    out = torch.full_like(src, OUT_FILL)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream().cuda_stream
    assert B.op_run_noalloc(src.data_ptr(), out.data_ptr(), 130, 90, stride, 4, 6, 20, LIT,
                            s) == B.OP_OK
    assert_same(out.cpu().numpy(), cpu_filter(buf, 130, 90, stride, 4, 6, 20, LIT), 130, 90,
                stride, 4, "noalloc literal")
    assert B.op_run_noalloc(src.data_ptr(), out.data_ptr(), 130, 90, stride, 4, 6, 255, LIT,
                            s) == B.OP_E_INVALID
    assert B.op_run_noalloc(src.data_ptr(), out.data_ptr(), 130, 90, stride, 4, 6, 20, 8,
                            s) == B.OP_E_INVALID  # unknown flag bit
    with pytest.raises(B.OilPaintError):
        OilPaint(130, 90, 6, 255, bpp=4, stride=stride, flags=LIT)
