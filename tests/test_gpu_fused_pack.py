"""The fused pack (OP_FUSED_PACK: 4-byte pixels read by the filter's halo
copies and packed in shared memory) against the pack prepass and the CPU
oracle, byte for byte, on every kernel path and word format."""
import numpy as np
import pytest
import torch

import __graft_entry__
import oracle
from paper_1405_1020_gb300 import binding as B
from paper_1405_1020_gb300 import synth
from paper_1405_1020_gb300.filter import OilPaint
from tests.pins import OUT_FILL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    __graft_entry__.build()
    torch.cuda.set_device(0)


def _run(buf, w, h, stride, r, L, flags, config, offset=0):
    """Filter through op_run; `offset` bytes shift the input (and output)
    pointer off its 16-byte alignment."""
    n = buf.size
    src_store = torch.from_numpy(np.concatenate([np.zeros(offset, np.uint8), buf])).cuda()
    dst_store = torch.full((n + offset,), OUT_FILL, dtype=torch.uint8, device="cuda")
    src, dst = src_store[offset:], dst_store[offset:]
    op = OilPaint(w, h, r, L, bpp=4, stride=stride, flags=flags, config=config)
    op.run(src, dst)
    assert op.sync_status() == B.OP_OK
    cfg = op.config()
    op.close()
    return dst.cpu().numpy(), cfg


def _oracle(buf, w, h, stride, r, L, flags):
    out = np.full(buf.size, OUT_FILL, np.uint8)
    return oracle.oilpaint(buf, w, h, stride, 4, r, L, mode=flags & 3, out=out)


# (w, h, r, L, flags, config): every path and word format, widths that are
# not multiples of 4 (the copies' last group reaches past the row's last
# pixel), images narrower than one tile, halo rows wider than one 2-D copy
CASES = [
    (333, 77, 3, 20, 0, None),
    (1001, 203, 15, 20, 0, None),                                       # straight-line K = 4
    (1001, 203, 15, 20, 0, {"tile_w": 512, "cols_per_thread": 8, "path": 3, "chunk_rows": 2,
                             "prefetch": 1}),
    (514, 130, 7, 64, 0, {"tile_w": 128, "cols_per_thread": 2, "path": 2}),
    (514, 130, 15, 64, 0, {"tile_w": 96, "cols_per_thread": 1}),       # one column, format 0
    (517, 99, 1, 20, 0, {"tile_w": 192, "cols_per_thread": 2}),        # runtime K = 2
    (600, 140, 20, 32, 0, {"tile_w": 128, "cols_per_thread": 4}),      # r > 15: format 2
    (600, 140, 44, 20, 0, None),
    (402, 90, 5, 17, 0, {"tile_w": 64, "path": 1}),                   # column histograms
    (255, 64, 4, 256, 0, None),
    (9, 5, 2, 20, 0, None),                                            # narrower than a tile
    (3, 40, 6, 20, 0, None),
    (300, 60, 4, 20, B.OP_LEVEL_INTDIV3, None),
    (300, 60, 4, 20, B.OP_LITERAL, None),
    (300, 60, 4, 254, B.OP_LITERAL | B.OP_LEVEL_INTDIV3, None),
    (257, 33, 12, 32, 0, {"tile_w": 256, "cols_per_thread": 4, "path": 2}),
    (333, 77, 1, 64, 0, {"tile_w": 128, "chunk_rows": 8, "path": 4}),     # direct path:
    (301, 50, 2, 256, 0, {"tile_w": 64, "chunk_rows": 3, "path": 4}),     # entering rows only
    (203, 41, 0, 20, B.OP_LITERAL, {"tile_w": 64, "chunk_rows": 8, "path": 4}),
]


@pytest.mark.parametrize("w,h,r,L,flags,cfg", CASES)
@pytest.mark.parametrize("pad", [0, 32])
def test_fused_equals_prepass_and_oracle(w, h, r, L, flags, cfg, pad):
    img = synth.camera_like(h, w, seed=w * 7 + h + r, npoly=max(4, w * h // 4000),
                            rad_range=(3, max(6, w // 4)))
    stride = (4 * w + 15) // 16 * 16 + pad
    buf, _ = synth.to_strided(img, bpp=4, stride=stride, alpha=77)
    want = _oracle(buf, w, h, stride, r, L, flags)
    fused, c1 = _run(buf, w, h, stride, r, L, flags | B.OP_FUSED_PACK, cfg)
    pre, c2 = _run(buf, w, h, stride, r, L, flags, cfg)
    assert c1 == c2
    assert np.array_equal(pre, want), "prepass differs from the oracle"
    assert np.array_equal(fused, want), "fused pack differs from the oracle"


@pytest.mark.parametrize("offset", [4, 8])
def test_unaligned_input_takes_the_prepass(offset):
    w, h, r, L = 301, 50, 6, 20
    img = synth.camera_like(h, w, seed=offset, npoly=10, rad_range=(3, 60))
    stride = 4 * w + 12  # a multiple of 4 bytes, not of 16
    buf, _ = synth.to_strided(img, bpp=4, stride=stride)
    want = _oracle(buf, w, h, stride, r, L, 0)
    got, _ = _run(buf, w, h, stride, r, L, B.OP_FUSED_PACK, None, offset=offset)
    assert np.array_equal(got, want)
    stride = 4 * w + 4 * (-w % 4)  # a multiple of 16 bytes, pointer shifted
    buf, _ = synth.to_strided(img, bpp=4, stride=stride)
    got, _ = _run(buf, w, h, stride, r, L, B.OP_FUSED_PACK, None, offset=offset)
    assert np.array_equal(got, _oracle(buf, w, h, stride, r, L, 0))


def test_rgb_ignores_the_flag():
    w, h, r, L = 203, 61, 5, 20
    img = synth.camera_like(h, w, seed=5, npoly=10, rad_range=(3, 60))
    buf, stride = synth.to_strided(img, bpp=3)
    src = torch.from_numpy(buf).cuda()
    dst = torch.full_like(src, OUT_FILL)
    op = OilPaint(w, h, r, L, bpp=3, stride=stride, flags=B.OP_FUSED_PACK)
    op.run(src, dst)
    assert op.sync_status() == B.OP_OK
    op.close()
    want = oracle.oilpaint(buf, w, h, stride, 3, r, L, out=np.full(buf.size, OUT_FILL, np.uint8))
    assert np.array_equal(dst.cpu().numpy(), want)


def test_fused_run_leaves_the_packed_workspace_alone():
    """With a caller-owned workspace filled with a marker: the fused run
    writes none of it, the prepass run writes the packed image there."""
    w, h, r, L = 640, 96, 9, 20
    img = synth.camera_like(h, w, seed=3, npoly=12, rad_range=(5, 80))
    buf, stride = synth.to_strided(img, bpp=4)
    src = torch.from_numpy(buf).cuda()
    want = _oracle(buf, w, h, stride, r, L, 0)
    for flags, untouched in ((B.OP_FUSED_PACK, True), (0, False)):
        op = OilPaint(w, h, r, L, bpp=4, stride=stride, flags=flags)
        n = B.op_workspace_size(op.handle)
        ws = torch.full((n,), 0xA5, dtype=torch.uint8, device="cuda")
        B.check(B.op_set_workspace(op.handle, ws.data_ptr(), n), "op_set_workspace")
        dst = torch.full_like(src, OUT_FILL)
        op.run(src, dst)
        assert op.sync_status() == B.OP_OK
        assert np.array_equal(dst.cpu().numpy(), want)
        assert bool((ws == 0xA5).all()) == untouched
        op.close()


def test_fused_host_pipeline_alternating_buffers():
    """op_run_host_async alternates two staging buffers: the two cached input
    maps must each follow their own pointer."""
    w, h, r, L = 800, 120, 15, 20
    imgs = [synth.camera_like(h, w, seed=s, npoly=20, rad_range=(5, 100)) for s in range(5)]
    bufs = [synth.to_strided(im, bpp=4)[0] for im in imgs]
    stride = 4 * w
    op = OilPaint(w, h, r, L, bpp=4, stride=stride, flags=B.OP_FUSED_PACK)
    outs = [np.full(b.size, OUT_FILL, np.uint8) for b in bufs]
    for b, o in zip(bufs, outs):
        op.run_host_async(b, o)
    assert op.sync_status() == B.OP_OK
    op.close()
    for b, o in zip(bufs, outs):
        assert np.array_equal(o, _oracle(b, w, h, stride, r, L, 0))
