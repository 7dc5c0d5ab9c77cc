"""Run one workload a few times, for profilers (ncu) to capture.

    python -m paper_1405_1020_gb300.profile_run image --radius 15 --levels 64 --reps 3
    python -m paper_1405_1020_gb300.profile_run batch --reps 3

`image`: the 4000x3000 RGBA-stride camera-like image (seed 2) with the
committed tuning table's (or the given) launch configuration.  `batch`: the
64-image mixed batch of the batch benchmark (log-uniform 320x240..4000x3000,
r in {2,4,8,12,20}, L in {16,20,32}), one graph launch per repetition.  Every
run is checked for device errors; nothing is timed.
"""
from __future__ import annotations

import argparse
import json
import sys

import torch

from . import binding as B
from . import synth
from .filter import Batch, OilPaint, load_tuning


def run_image(radius: int, levels: int, reps: int, config: dict | None) -> dict:
    img = synth.camera_like(3000, 4000, seed=2)
    buf, stride = synth.to_strided(img, bpp=4, stride=16000)
    src = torch.from_numpy(buf).cuda()
    dst = torch.empty_like(src)
    op = OilPaint(4000, 3000, radius, levels, bpp=4, stride=stride, config=config)
    for _ in range(reps):
        op.run(src, dst)
    if op.sync_status() != B.OP_OK:
        raise RuntimeError("device error")
    cfg = op.config()
    op.close()
    return cfg


def run_batch(reps: int) -> dict:
    from .batchbench import make_batch, make_pool
    images = make_batch(synth.batch_specs(n=64), make_pool())
    pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
    b = Batch(64, pix + 4096, max(im["r"] for im in images), max(im["L"] for im in images))
    outs = [torch.empty_like(im["src"]) for im in images]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    b.set([(im["src"], o, im["w"], im["h"], im["stride"], 3, im["r"], im["L"])
           for im, o in zip(images, outs)], stream)
    b.capture(stream)
    for _ in range(reps):
        b.launch_graph(stream)
    if b.sync_status(stream) != B.OP_OK:
        raise RuntimeError("device error")
    cfg = b.config()
    b.close()
    return cfg


def main(argv=None) -> int:
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("what", choices=["image", "batch"])
    p.add_argument("--radius", type=int, default=15)
    p.add_argument("--levels", type=int, default=20)
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--config", default=None, help="launch config JSON (image only)")
    args = p.parse_args(argv)
    import __graft_entry__
    __graft_entry__.build()
    load_tuning()
    if args.what == "image":
        cfg = run_image(args.radius, args.levels, args.reps,
                        json.loads(args.config) if args.config else None)
    else:
        cfg = run_batch(args.reps)
    print(json.dumps({"what": args.what, "config": cfg}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
