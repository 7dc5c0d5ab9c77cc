"""Randomized parity campaign, run by hand on a GPU (not collected by pytest):

    python tests/fuzz_campaign.py SEED SECONDS [image|batch]

Draws configurations from seven families -- the default choice at any
radius and level count, one column per thread, difference histograms with
the radius at run time, the straight-line paths, column histograms, the
direct path, and the tuned table's entries -- with random image sizes
(1..1200 x 1..300), 3 or 4 bytes per pixel, row padding, both level modes,
literal mode, the fused pack, tile heights, halo chunk heights and prefetch
depths, camera-like images with runs of white; filters each through op_run
and compares every byte with the oracle.  A configuration the library
refuses must be refused with OP_E_UNSUPPORTED.  `batch` runs random image
sets through the batch API instead.  Exits 1 on any difference.
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import numpy as np
import __graft_entry__
__graft_entry__.build()
import torch
import oracle
from paper_1405_1020_gb300 import binding as B, synth
from paper_1405_1020_gb300.filter import OilPaint, load_tuning
load_tuning()
FILL = 0x5A
rng = np.random.default_rng(int(sys.argv[1]) if len(sys.argv) > 1 else 1234)
budget = float(sys.argv[2]) if len(sys.argv) > 2 else 480.0
MODE = sys.argv[3] if len(sys.argv) > 3 else "image"


def batch_campaign():
    """Random batches (1..40 images of mixed size, radius, levels, bytes per
    pixel and mode) through op_batch_set, run eagerly and replayed from the
    captured graph, every image against the oracle."""
    from paper_1405_1020_gb300.filter import Batch
    t0 = time.time(); nb = ni = 0; fails = []
    stream = torch.cuda.Stream()
    while time.time() - t0 < budget:
        n = int(rng.integers(1, 41))
        ims = []
        for _ in range(n):
            w = int(rng.integers(1, 700)); h = int(rng.integers(1, 300))
            bpp = int(rng.choice([3, 4])); mode = int(rng.choice([0, 1, B.OP_LITERAL]))
            r = int(rng.choice([0, 1, 2, 3, 5, 8, 12, 15, 16, 20, 31, 44]))
            L = int(rng.choice([1, 2, 7, 16, 20, 21, 32, 33, 64, 200, 254]))
            img = synth.camera_like(h, w, seed=int(rng.integers(1 << 30)), npoly=8,
                                    rad_range=(1, max(2, w // 3)))
            if rng.random() < 0.3:
                img[rng.random((h, w)) < 0.2] = 255
            buf, stride = synth.to_strided(img, bpp=bpp, stride=w * bpp + int(rng.integers(0, 9)))
            src = torch.from_numpy(buf).cuda()
            ims.append(dict(buf=buf, src=src, dst=torch.full_like(src, FILL), w=w, h=h,
                            stride=stride, bpp=bpp, r=r, L=L, mode=mode))
        torch.cuda.synchronize()
        pix = Batch.padded_pixels([(im["w"], im["h"]) for im in ims])
        b = Batch(n, pix + 4096, max(im["r"] for im in ims), max(im["L"] for im in ims))
        descs = [(im["src"], im["dst"], im["w"], im["h"], im["stride"], im["bpp"], im["r"],
                  im["L"], im["mode"]) for im in ims]
        for how in ("eager", "graph"):
            for im in ims:
                im["dst"].fill_(FILL)
            torch.cuda.synchronize()
            b.set(descs, stream)
            if how == "eager":
                b.run(stream)
            else:
                b.capture(stream)
                b.launch_graph(stream)
            st = b.sync_status(stream)
            for k, im in enumerate(ims):
                want = oracle.oilpaint(im["buf"], im["w"], im["h"], im["stride"], im["bpp"],
                                       im["r"], im["L"], mode=im["mode"],
                                       out=np.full(im["buf"].size, FILL, np.uint8))
                if st != B.OP_OK or not np.array_equal(im["dst"].cpu().numpy(), want):
                    fails.append(dict(how=how, k=k, n=n, w=im["w"], h=im["h"], r=im["r"],
                                      L=im["L"], bpp=im["bpp"], mode=im["mode"], status=st))
                    print("FAIL", fails[-1], flush=True)
                ni += 1
        b.close()
        nb += 1
    print(json.dumps({"batches": nb, "images": ni, "failures": len(fails),
                      "seconds": round(time.time() - t0, 1)}))
    sys.exit(1 if fails else 0)


if MODE == "batch":
    batch_campaign()
t0 = time.time(); n = 0; refused = 0; fails = []
while time.time() - t0 < budget:
    fam = int(rng.integers(0, 7))
    w = int(rng.choice([1, 2, 7, 31, 64, 100, 129, 257, 513, int(rng.integers(1, 1200))]))
    h = int(rng.choice([1, 2, 3, 9, 40, int(rng.integers(1, 300))]))
    bpp = int(rng.choice([3, 4])); pad = int(rng.choice([0, 1, 3, 4, 12, 16]))
    mode = int(rng.choice([0, 1, B.OP_LITERAL, B.OP_LITERAL | 1]))
    flags = mode | (B.OP_FUSED_PACK if rng.random() < 0.25 else 0)
    Lmax = 254 if mode & B.OP_LITERAL else 256
    cfg = None
    if fam == 0:    # default configuration, any r, L
        r = int(rng.integers(0, 45)); L = int(rng.integers(1, Lmax + 1))
    elif fam == 1:  # one column per thread
        r = int(rng.integers(0, 45)); L = int(rng.integers(1, Lmax + 1))
        cfg = {"tile_w": int(rng.choice([32, 64, 96, 128])), "cols_per_thread": 1, "path": 0}
    elif fam == 2:  # runtime K columns
        r = int(rng.integers(0, 45)); L = int(rng.integers(1, 33)); K = int(rng.choice([2, 4]))
        cfg = {"tile_w": int(rng.choice([32, 64, 96, 128])) * K, "cols_per_thread": K, "path": 0}
    elif fam == 3:  # straight-line
        K = int(rng.choice([2, 4, 8])); r = int(rng.integers({2: 1, 4: 2, 8: 4}[K], 16))
        L = int(rng.integers(1, (65 if K == 2 else 33)))
        path = 2 if K == 2 else int(rng.choice([2, 3]))
        cfg = {"tile_w": int(rng.choice([32, 64])) * K, "cols_per_thread": K, "path": path}
    elif fam == 4:  # column histograms
        r = int(rng.integers(0, 45)); L = int(rng.integers(1, 33)); twk = int(rng.choice([1, 2]))
        cfg = {"tile_w": int(rng.choice([32, 64, 128])) * twk, "cols_per_thread": twk, "path": 1}
    elif fam == 5:  # direct
        r = int(rng.integers(0, 3)); L = int(rng.integers(1, Lmax + 1))
        cfg = {"tile_w": int(rng.choice([32, 64, 96, 128])), "cols_per_thread": 1, "path": 4}
    else:           # tuned table entries
        r = int(rng.choice([0, 1, 2, 4, 8, 12, 15, 20])); L = int(rng.choice([16, 20, 32, 64, 256]))
    if cfg is not None:
        cfg.update({"tile_h": int(rng.choice([0, 0, 1, 5, 33])), "chunk_rows": int(rng.choice([1, 2, 3, 4, 8])),
                    "prefetch": int(rng.integers(1, 3))})
    L = min(L, Lmax)
    img = synth.camera_like(h, w, seed=int(rng.integers(1 << 30)), npoly=int(rng.integers(1, 30)),
                            rad_range=(1, max(2, w // 3)), noise=float(rng.choice([0.0, 3.0, 8.0])))
    if rng.random() < 0.3:
        img[rng.random((h, w)) < rng.random() * 0.5] = 255
    stride = w * bpp + pad
    if flags & B.OP_FUSED_PACK and bpp == 4 and rng.random() < 0.7:
        stride = (4 * w + 15) // 16 * 16 + 16 * int(rng.integers(0, 2))
    buf, stride = synth.to_strided(img, bpp=bpp, stride=stride)
    try:
        op = OilPaint(w, h, r, L, bpp=bpp, stride=stride, flags=flags, config=cfg)
    except B.OilPaintError as e:
        assert e.status == B.OP_E_UNSUPPORTED, (e.status, w, h, r, L, cfg)
        refused += 1; continue
    src = torch.from_numpy(buf).cuda(); dst = torch.full_like(src, FILL)
    op.run(src, dst); st = op.sync_status(); got_cfg = op.config(); op.close()
    want = oracle.oilpaint(buf, w, h, stride, bpp, r, L, mode=mode, out=np.full(buf.size, FILL, np.uint8))
    got = dst.cpu().numpy()
    n += 1
    if st != B.OP_OK or not np.array_equal(got, want):
        fails.append(dict(w=w, h=h, r=r, L=L, bpp=bpp, stride=stride, flags=flags, cfg=got_cfg, status=st,
                          diff=int((got != want).sum())))
        print("FAIL", fails[-1], flush=True)
print(json.dumps({"cases": n, "refused": refused, "failures": len(fails), "seconds": round(time.time() - t0, 1)}))
sys.exit(1 if fails else 0)
