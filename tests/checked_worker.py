"""Runs every kernel path through the bounds-checking build and compares each
result with the oracle; exits 0 only if all match and no check fired.

Started by tests/test_gpu_checked.py in a child process with
OPK_LIBRARY=checked (the binding loads one library per process)."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1405_1020_gb300 import binding as B  # noqa: E402
from paper_1405_1020_gb300 import synth  # noqa: E402
from paper_1405_1020_gb300.filter import Batch, OilPaint  # noqa: E402

FILL = 0x5A


def want(buf, w, h, stride, bpp, r, L, mode):
    out = np.full(buf.size, FILL, np.uint8)
    return oracle.oilpaint(buf, w, h, stride, bpp, r, L, mode=mode, out=out)


def image(w, h, bpp, seed, stride=None):
    img = synth.camera_like(h, w, seed=seed, npoly=15, rad_range=(2, 60))
    img[np.random.default_rng(seed).random((h, w)) < 0.1] = 255
    return synth.to_strided(img, bpp=bpp, stride=stride or w * bpp + 4)


def main() -> int:
    assert B.LIB_PATH.endswith("liboilpaint_checked.so"), B.LIB_PATH
    torch.cuda.set_device(0)
    cases = [  # (r, L, mode, config)
        (15, 20, 0, {"tile_w": 256, "cols_per_thread": 8, "chunk_rows": 1}),
        (4, 32, 1, {"tile_w": 512, "cols_per_thread": 8, "chunk_rows": 2}),
        (11, 7, B.OP_LITERAL, {"tile_w": 256, "cols_per_thread": 8, "chunk_rows": 3}),
        (14, 20, 0, {"tile_w": 512, "cols_per_thread": 4, "chunk_rows": 1}),
        (15, 20, 0, {"tile_w": 128, "cols_per_thread": 4, "chunk_rows": 2, "path": 2}),
        (2, 32, B.OP_LITERAL, {"tile_w": 256, "cols_per_thread": 4, "chunk_rows": 1, "path": 3}),
        (9, 16, 1, {"tile_w": 256, "cols_per_thread": 8, "chunk_rows": 2, "path": 2}),
        (15, 64, 0, {"tile_w": 64, "cols_per_thread": 2, "chunk_rows": 2, "path": 2}),
        (1, 47, B.OP_LITERAL, {"tile_w": 128, "cols_per_thread": 2, "chunk_rows": 1, "path": 2}),
        (2, 20, 0, {"tile_w": 64, "cols_per_thread": 1}),
        (20, 64, 1, {"tile_w": 32, "cols_per_thread": 1}),
        (15, 20, 0, {"tile_w": 128, "cols_per_thread": 4, "chunk_rows": 2}),
        (9, 32, 0, {"tile_w": 128, "cols_per_thread": 2}),
        (30, 20, 1, {"tile_w": 64, "cols_per_thread": 2}),
        (20, 16, 0, {"tile_w": 128, "cols_per_thread": 4}),
        (15, 20, 0, {"tile_w": 128, "cols_per_thread": 1, "path": 1}),
        (25, 32, 0, {"tile_w": 128, "cols_per_thread": 2, "path": 1}),
        (6, 20, B.OP_LITERAL, {"tile_w": 128, "cols_per_thread": 4}),
        (17, 254, B.OP_LITERAL, {"tile_w": 32, "cols_per_thread": 1}),
        (1, 256, 0, {"tile_w": 128, "chunk_rows": 4, "path": 4}),
        (2, 64, B.OP_LITERAL, {"tile_w": 64, "chunk_rows": 3, "path": 4}),
        (2, 20, 1, {"tile_w": 96, "chunk_rows": 1, "prefetch": 2, "path": 4}),
    ]
    n = 0
    for k, (r, L, mode, cfg) in enumerate(cases):
        for bpp in (3, 4):
            buf, stride = image(233, 150, bpp, seed=k)
            src = torch.from_numpy(buf).cuda()
            dst = torch.full_like(src, FILL)
            op = OilPaint(233, 150, r, L, bpp=bpp, stride=stride, flags=mode, config=cfg)
            op.run(src, dst)
            st = op.sync_status()
            assert st == B.OP_OK, (r, L, cfg, B.status_string(st))
            op.close()
            assert np.array_equal(dst.cpu().numpy(), want(buf, 233, 150, stride, bpp, r, L, mode)), \
                (r, L, mode, bpp, cfg)
            n += 1
    # the fused pack (4-byte pixels on 16-byte rows; every path and word format)
    for k, (r, L, mode, cfg) in enumerate(cases):
        buf, stride = image(233, 150, 4, seed=200 + k, stride=944)
        src = torch.from_numpy(buf).cuda()
        dst = torch.full_like(src, FILL)
        op = OilPaint(233, 150, r, L, bpp=4, stride=stride, flags=mode | B.OP_FUSED_PACK,
                      config=cfg)
        op.run(src, dst)
        st = op.sync_status()
        assert st == B.OP_OK, (r, L, cfg, "fused", B.status_string(st))
        op.close()
        assert np.array_equal(dst.cpu().numpy(), want(buf, 233, 150, stride, 4, r, L, mode)), \
            (r, L, mode, "fused", cfg)
        n += 1
    # batch: all four groups (r above 15 or not x L above 20 or not), literal
    # and default images
    images = []
    for k in range(8):
        w, h = 100 + 37 * k, 60 + 11 * k
        buf, stride = image(w, h, 3, seed=50 + k)
        src = torch.from_numpy(buf).cuda()
        images.append((buf, src, torch.full_like(src, FILL), w, h, stride, [1, 8, 15, 16, 20, 3, 12, 20][k],
                       [20, 16, 32, 20, 32, 20, 16, 20][k], B.OP_LITERAL if k % 3 == 0 else 0))
    pix = Batch.padded_pixels([(im[3], im[4]) for im in images])
    b = Batch(8, pix + 64, 20, 32)
    torch.cuda.synchronize()
    b.set([(im[1], im[2], im[3], im[4], im[5], 3, im[6], im[7], im[8]) for im in images])
    b.run()
    st = b.sync_status()
    assert st == B.OP_OK, B.status_string(st)
    for buf, _, dst, w, h, stride, r, L, mode in images:
        assert np.array_equal(dst.cpu().numpy(), want(buf, w, h, stride, 3, r, L, mode)), (r, L)
        n += 1
    b.close()
    # the allocation-free entry point
    buf, stride = image(180, 90, 4, seed=99)
    src = torch.from_numpy(buf).cuda()
    dst = torch.full_like(src, FILL)
    torch.cuda.synchronize()
    st = B.op_run_noalloc(src.data_ptr(), dst.data_ptr(), 180, 90, stride, 4, 9, 20, 0,
                          torch.cuda.current_stream().cuda_stream)
    assert st == B.OP_OK, B.status_string(st)
    assert np.array_equal(dst.cpu().numpy(), want(buf, 180, 90, stride, 4, 9, 20, 0))
    n += 1
    print(f"checked build: {n} runs, all equal to the oracle, no bounds check fired")
    return 0


if __name__ == "__main__":
    sys.exit(main())
