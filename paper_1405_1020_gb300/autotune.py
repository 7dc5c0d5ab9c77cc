"""Launch-configuration autotuner.

For a (radius, levels) pair it times the filter kernel (CUDA events on the
launching stream, the pack prepass excluded through op_set_profile_event)
under every candidate configuration -- threads per CTA, output columns per
thread, halo chunk height, prefetch depth and tile height -- on a
synthetic camera-like image, checks that every candidate writes identical
bytes, and records the fastest in the library's tuning table
(op_tune_table_set), from which op_create and op_batch_set take it.

Results can be saved to / loaded from a JSON table keyed by
"<radius>,<levels>"; the committed table for GB300 is tuning_gb300.json.
"""
from __future__ import annotations

import itertools
import json
import os
import statistics

import torch

from . import binding as B
from .filter import OilPaint

TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")


def candidates(radius: int, levels: int, tile_hs=(0,)) -> list[dict]:
    """Threads per CTA x output columns per thread x halo chunk height x
    prefetch depth x tile height; configurations the library refuses (halo
    wider than 256 columns, shared memory) are skipped when timed."""
    out = []
    for nt, cpt, ch, pf, th in itertools.product((32, 64, 96, 128), (1, 2, 4), (1, 2, 4, 8, 16), (1, 2),
                                                  tile_hs):
        out.append({"tile_w": nt * cpt, "tile_h": th, "chunk_rows": ch, "prefetch": pf,
                    "cols_per_thread": cpt, "path": 0})
    if levels <= 32:  # column histograms, levels across lanes
        for nt, cpt, ch, pf, th in itertools.product((32, 64, 128), (1, 2), (1, 2, 4), (1, 2),
                                                      tile_hs):
            out.append({"tile_w": nt * cpt, "tile_h": th, "chunk_rows": ch, "prefetch": pf,
                        "cols_per_thread": cpt, "path": 1})
    return out


def _time_filter(op: OilPaint, src, dst, reps: int) -> float:
    stream = torch.cuda.current_stream()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps)]
    for e in evs:
        e[0].record(stream)
    op.run(src, dst)  # warm-up under this configuration
    times = []
    for e0, e1 in evs:
        B.check(B.op_set_profile_event(op.handle, e0.cuda_event), "profile event")
        op.run(src, dst)
        e1.record(stream)
    torch.cuda.synchronize()
    B.op_set_profile_event(op.handle, None)
    for e0, e1 in evs:
        times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def tune_image(width: int, height: int, bpp: int, stride: int, radius: int, levels: int,
               src: torch.Tensor | None = None, flags: int = B.OP_LEVEL_PAPER, reps: int = 5,
               tile_hs=(0,), record: bool = True, verbose: bool = False) -> dict:
    """Search the candidates on one image (a seeded camera-like image unless
    `src` is given); returns {"config", "ms", "results"}."""
    if src is None:
        from . import synth
        img = synth.camera_like(height, width, seed=2)
        buf, stride = synth.to_strided(img, bpp=bpp, stride=stride)
        src = torch.from_numpy(buf).cuda()
    dst = torch.empty_like(src)
    ref = None
    results = []
    op = OilPaint(width, height, radius, levels, bpp=bpp, stride=stride, flags=flags)
    try:
        for cfg in candidates(radius, levels, tile_hs):
            try:
                op.set_config(cfg)
            except B.OilPaintError as e:
                if e.status == B.OP_E_UNSUPPORTED:
                    continue
                raise
            ms = _time_filter(op, src, dst, reps)
            if op.sync_status() != B.OP_OK:
                raise B.OilPaintError(f"device error under {cfg}")
            if ref is None:
                ref = dst.clone()
            elif not torch.equal(ref, dst):
                raise B.OilPaintError(f"config {cfg} changed the output")
            results.append({"config": cfg, "ms": ms, "tile_h_used": op.config()["tile_h"]})
            if verbose:
                print(f"{cfg} {ms:.4f} ms")
    finally:
        op.close()
    results.sort(key=lambda r: r["ms"])
    best = results[0]
    if record:
        B.check(B.op_tune_table_set(radius, levels, B.op_config_t.make(**best["config"])),
                "op_tune_table_set")
    return {"config": best["config"], "ms": best["ms"], "results": results}


def load_table(path: str = TABLE_PATH) -> int:
    """Load a saved table into the library's tuning table; returns its size."""
    from .filter import load_tuning
    return load_tuning(path)


def save_table(entries: dict, path: str, device_name: str) -> None:
    with open(path, "w") as f:
        json.dump({"device": device_name, "entries": entries}, f, indent=1, sort_keys=True)


def tune_pairs(pairs, width: int = 4000, height: int = 3000, bpp: int = 4, reps: int = 5,
               path: str | None = None, verbose: bool = False) -> dict:
    """Tune every (radius, levels) pair on a width x height image and
    optionally save the table."""
    from . import synth
    img = synth.camera_like(height, width, seed=2)
    buf, stride = synth.to_strided(img, bpp=bpp)
    src = torch.from_numpy(buf).cuda()
    entries = {}
    for r, L in pairs:
        res = tune_image(width, height, bpp, stride, r, L, src=src, reps=reps, verbose=verbose)
        entries[f"{r},{L}"] = {"config": res["config"], "ms": res["ms"],
                               "image": f"{width}x{height} bpp={bpp}"}
    if path:
        save_table(entries, path, torch.cuda.get_device_name())
    return entries
