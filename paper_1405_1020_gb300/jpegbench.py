"""Timing of the decode -> filter -> encode pipeline (section 3.2's
ApplyOilPaintOnFile, on byte buffers) on one image.

The input is a synthetic camera-like RGB image encoded once by the pipeline's
own encoder; each timed call decodes it, filters it and encodes the result.
Reported: wall time per call (host clock around op_jpeg_filter, which returns
after the encoded bytes are on the host) and the three phase times from the
library's CUDA events, medians over the timed calls; and the throughput of a
JpegPool of `workers` host threads (a codec context and stream each, created
before the timed region) over `images` copies of the image, each thread
taking `batch` images per op_jpeg_filter_batch call (one batched decode on
the GPU's JPEG engines), best of two passes.
"""
from __future__ import annotations

import statistics
import time

import numpy as np


def run(width: int = 4000, height: int = 3000, radius: int = 15, levels: int = 20,
        quality: int = 90, calls: int = 10, warmup: int = 2, seed: int = 2,
        workers: int = 4, batch: int = 8, images: int = 64) -> dict:
    import torch

    from . import jpeg as J
    from . import synth
    from .csrc import build as cbuild

    try:
        built = cbuild.build_jpeg()
    except Exception as e:  # noqa: BLE001 -- the benchmark line reports it
        return {"unavailable": f"liboilpaint_jpeg.so did not build: {e}"}
    if built is None or not J.available():
        return {"unavailable": "nvJPEG is not in this CUDA toolkit"}
    src = synth.camera_like(height, width, seed=seed)
    rgb = torch.from_numpy(np.ascontiguousarray(src).reshape(height, 3 * width)).cuda()
    with J.JpegPipeline() as p:
        data = p.encode(rgb, width, height, quality=quality, sampling=J.OP_JPEG_CSS_420)
        for _ in range(warmup):
            p.filter(data, radius, levels, quality=quality)
        walls, phases = [], []
        for _ in range(calls):
            t = time.perf_counter()
            out = p.filter(data, radius, levels, quality=quality)
            walls.append(time.perf_counter() - t)
            phases.append(p.last_timing())
        many = [data] * images
        with J.JpegPool(workers, batch) as pool:
            pool.filter_many(many[:workers * batch], radius, levels, quality=quality)  # contexts
            many_s = float("inf")
            for _ in range(2):
                t = time.perf_counter()
                outs = pool.filter_many(many, radius, levels, quality=quality)
                many_s = min(many_s, time.perf_counter() - t)
                if any(o != out for o in outs):
                    raise RuntimeError("filter_many output differs from filter")
    wall = statistics.median(walls)
    med = {k: round(statistics.median(ph[k] for ph in phases), 4) for k in phases[0]}
    return {
        "threads": {"workers": workers, "batch": batch, "images": len(many),
                    "ms_per_image": round(many_s / len(many) * 1e3, 3),
                    "mpix_s": round(len(many) * width * height / many_s / 1e6, 1)},
        "workload": f"{width}x{height} camera-like RGB, JPEG q{quality} 4:2:0 in and out, "
                    f"r={radius} L={levels}",
        "calls": calls, "ms_per_image": round(wall * 1e3, 3),
        "mpix_s": round(width * height / wall / 1e6, 1),
        "phase_ms": med, "jpeg_in_bytes": len(data), "jpeg_out_bytes": len(out),
        "codec": "nvJPEG: one call's decode with Huffman decoding on the host, the rest on "
                 "the GPU; batched decode on the GPU's JPEG engines",
    }
