"""Radius sweep of the 1920x1080 blobs image (seed 1, RGB, L = 20, r = 1..10).

    python -m paper_1405_1020_gb300.sweep [--steps 50] [--radii 1-10]

For every radius: pack + filter time per image (CUDA events around op_run on
the launching stream, a 512 MiB write between steps to flush L2, the
committed tuning table's configuration), Mpix/s, the filter's share, and two
rooflines: the filter against the integer-ALU peak of the method's op count
(16r + L + 11 per pixel, 152 SMs x 128 lanes x the SM clock), and the whole
step against HBM with the algorithmic bytes only -- 3 bytes read and 3
written per RGB pixel; the packed words' round trip (4 + 4 bytes per pixel)
is a choice of this implementation, not work the method needs, so it is
reported beside (`moved_bytes_frac`), not counted.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys

import torch

from . import binding as B
from . import synth
from .filter import OilPaint, load_tuning

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INT_LANES_PER_SM = 128


def _peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def run(radii=range(1, 11), steps: int = 50, warmup: int = 5, levels: int = 20) -> dict:
    h, w = 1080, 1920
    buf, stride = synth.to_strided(synth.blobs_rgb(h, w, seed=1), bpp=3)
    src = torch.from_numpy(buf).cuda()
    dst = torch.empty_like(src)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    peaks = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    hbm = float(peaks.get("hbm_gbs", 6689.8))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    int_peak = sms * INT_LANES_PER_SM * sm_mhz * 1e6
    rows = []
    for r in radii:
        op = OilPaint(w, h, r, levels, bpp=3, stride=stride)
        step_ms, filt_ms = [], []
        for it in range(warmup + steps):
            flush.fill_(it & 0xFF)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e1.record(stream)  # marks it recorded; the library records it again
            e0.record(stream)
            B.check(B.op_set_profile_event(op.handle, e1.cuda_event), "op_set_profile_event")
            op.run(src, dst)
            e2.record(stream)
            torch.cuda.synchronize()
            if it >= warmup:
                step_ms.append(e0.elapsed_time(e2))
                filt_ms.append(e1.elapsed_time(e2))
        if op.sync_status() != B.OP_OK:
            raise RuntimeError(f"device error at r={r}")
        cfg = op.config()
        op.close()
        ms, fms = statistics.median(step_ms), statistics.median(filt_ms)
        px = w * h
        ops = 16 * r + levels + 11
        rows.append({
            "r": r, "ms": round(ms, 4), "filter_ms": round(fms, 4),
            "mpix_s": round(px / ms / 1e3, 1),
            "alu_frac": round(ops * px / (fms / 1e3) / int_peak, 4),
            "hbm_frac": round((3 + 3) * px / (ms / 1e3) / (hbm * 1e9), 4),
            "moved_bytes_frac": round((3 + 3 + 4 + 4) * px / (ms / 1e3) / (hbm * 1e9), 4),
            "config": {k: cfg[k] for k in ("tile_w", "chunk_rows", "cols_per_thread", "path")},
        })
    return {"workload": "1920x1080 blobs RGB (seed 1), L=20", "steps": steps,
            "l2": "flushed between steps (512 MiB write)", "sweep": rows}


def _parse_radii(text: str) -> list[int]:
    if "-" in text:
        a, b = (int(v) for v in text.split("-"))
        return list(range(a, b + 1))
    return [int(v) for v in text.split(",")]


def main(argv=None) -> int:
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--radii", default="1-10")
    args = p.parse_args(argv)
    import __graft_entry__
    __graft_entry__.build()
    load_tuning()
    print(json.dumps(run(_parse_radii(args.radii), args.steps, args.warmup)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
