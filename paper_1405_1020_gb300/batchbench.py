"""The mixed-batch workload: many images of uneven sizes and radii filtered
by one persistent launch (replayed from a CUDA graph) against one plain
op_run per image on the same stream, with identical outputs required.

Images: `batch_specs` (64 images, pixel counts log-uniform in
[320x240, 4000x3000], aspect 4:3 or 16:9, radius uniform in {2,4,8,12,20},
L uniform in {16,20,32}); their pixels are crops of two seeded camera-like
4800x3600 images, RGB with packed rows.
"""
from __future__ import annotations

import statistics

import numpy as np
import torch

from . import binding as B
from . import synth
from .filter import Batch, OilPaint

POOL_H, POOL_W = 3600, 4800


def make_pool(seeds=(31, 32)):
    return [synth.camera_like(POOL_H, POOL_W, seed=s) for s in seeds]


def make_batch(specs, pool):
    images = []
    rng = np.random.default_rng(7)
    for i, sp in enumerate(specs):
        src = pool[i % len(pool)]
        w, h = min(sp.width, POOL_W), min(sp.height, POOL_H)
        y0 = int(rng.integers(0, POOL_H - h + 1))
        x0 = int(rng.integers(0, POOL_W - w + 1))
        crop = np.ascontiguousarray(src[y0:y0 + h, x0:x0 + w])
        buf, stride = synth.to_strided(crop, bpp=3)
        images.append(dict(w=w, h=h, stride=stride, r=sp.radius, L=sp.levels,
                           src=torch.from_numpy(buf).cuda()))
    return images


def _time(fn, steps, stream):
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for e0, e1 in evs:
        e0.record(stream)
        fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return [e0.elapsed_time(e1) for e0, e1 in evs]


def run(steps: int = 10, warmup: int = 3, n: int = 64, config=None) -> dict:
    """Times both forms on the same stream; returns the summary dict."""
    specs = synth.batch_specs(n=n)
    images = make_batch(specs, make_pool())
    total_px = sum(im["w"] * im["h"] for im in images)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()  # uploads on the default stream are complete
    with torch.cuda.stream(stream):
        # plain: one op per image (each with its tuned or default config)
        ops = [OilPaint(im["w"], im["h"], im["r"], im["L"], bpp=3, stride=im["stride"])
               for im in images]
        plain_out = [torch.empty_like(im["src"]) for im in images]

        def plain():
            for op, im, o in zip(ops, images, plain_out):
                op.run(im["src"], o, stream)

        # batched: one persistent launch over all tiles of all images
        max_r = max(im["r"] for im in images)
        max_L = max(im["L"] for im in images)
        pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
        batch = Batch(n, pix + 4096, max_r, max_L, config=config)
        batch_out = [torch.empty_like(im["src"]) for im in images]
        batch.set([(im["src"], o, im["w"], im["h"], im["stride"], 3, im["r"], im["L"])
                   for im, o in zip(images, batch_out)], stream)
        batch.capture(stream)

        def batched():
            batch.launch_graph(stream)

        def batched_eager():
            batch.run(stream)

        for _ in range(warmup):
            plain()
            batched()
            batched_eager()
        stream.synchronize()
        t_plain = _time(plain, steps, stream)
        t_graph = _time(batched, steps, stream)
        t_eager = _time(batched_eager, steps, stream)
    if batch.sync_status(stream) != B.OP_OK or any(op.sync_status(stream) for op in ops):
        raise RuntimeError("device error in the batched workload")
    identical = all(torch.equal(a, b) for a, b in zip(plain_out, batch_out))
    if not identical:
        raise RuntimeError("batched and plain outputs differ")
    ms_plain = statistics.median(t_plain)
    ms_graph = statistics.median(t_graph)
    ms_eager = statistics.median(t_eager)
    cfg = batch.config()
    groups = batch.groups()
    for op in ops:
        op.close()
    batch.close()
    return {
        "workload": f"{n} camera-like RGB images, log-uniform 320x240..4000x3000, "
                    "r in {2,4,8,12,20}, L in {16,20,32}",
        "images": n, "mpix": round(total_px / 1e6, 3), "steps": steps,
        "plain_ms": round(ms_plain, 3), "batched_graph_ms": round(ms_graph, 3),
        "batched_eager_ms": round(ms_eager, 3),
        "plain_mpix_s": round(total_px / ms_plain / 1e3, 1),
        "batched_mpix_s": round(total_px / ms_graph / 1e3, 1),
        "speedup_vs_plain": round(ms_plain / ms_graph, 3),
        "launches_plain": 2 * n, "launches_batched": 1 + len(groups),
        "identical_outputs": identical, "config": cfg,
        "groups": [{"max_radius": g["max_radius"], "max_levels": g["max_levels"],
                    **{k: g["config"][k] for k in ("tile_w", "chunk_rows", "cols_per_thread")}}
                   for g in groups],
    }



def tune(table_path: str | None = None, n: int = 64, reps: int = 7, verbose: bool = True) -> dict:
    """Tunes the batch groups' configurations on this workload
    (autotune.tune_batch, coordinate descent over the groups) and writes
    them as the batch entries of the tuning table (the single-image entries
    are kept)."""
    import json

    from . import autotune
    from .filter import load_tuning

    path = table_path or autotune.TABLE_PATH
    load_tuning(path)
    images = make_batch(synth.batch_specs(n=n), make_pool())
    for im in images:
        im["bpp"] = 3
    max_r = max(im["r"] for im in images)
    max_L = max(im["L"] for im in images)
    res = autotune.tune_batch(images, max_r, max_L, reps=reps, verbose=verbose)
    with open(path) as f:
        table = json.load(f)
    workload = "64-image mixed batch, r in {2,4,8,12,20}, L in {16,20,32}"
    table["batch_entries"] = {k: {"batch_ms": round(res["ms"], 4), "config": v["config"],
                                  "workload": workload}
                              for k, v in res["groups"].items()}
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
        f.write("\n")
    return res


if __name__ == "__main__":
    import argparse
    import json
    import sys

    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--tune", action="store_true", help="tune the batch groups and save the table")
    p.add_argument("--steps", type=int, default=10)
    a = p.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    from .filter import load_tuning
    if a.tune:
        r = tune()
        print(json.dumps({"untuned_ms": r["ms_untuned"], "tuned_ms": r["ms"],
                          "groups": r["groups"]}))
    load_tuning()
    print(json.dumps(run(steps=a.steps)))
    sys.exit(0)
