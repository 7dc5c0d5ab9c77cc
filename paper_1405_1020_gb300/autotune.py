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
    prefetch depth x tile height, on every path that applies; configurations
    the library refuses (shared memory, a path outside its radius range) are
    skipped when timed."""
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
    if levels <= 64 and 1 <= radius <= 15:  # straight-line, two columns per thread
        for nt, ch, pf, th in itertools.product((32, 64), (1, 2, 4), (1, 2), tile_hs):
            out.append({"tile_w": nt * 2, "tile_h": th, "chunk_rows": ch, "prefetch": pf,
                        "cols_per_thread": 2, "path": 2})
    if 0 <= radius <= 2:  # direct: windows in registers, levels compared pairwise
        for nt, ch, pf, th in itertools.product((64, 128), (2, 4, 8), (1, 2), tile_hs):
            out.append({"tile_w": nt, "tile_h": th, "chunk_rows": ch, "prefetch": pf,
                        "cols_per_thread": 1, "path": 4})
    if levels <= 32 and 2 <= radius <= 15:  # straight-line difference histograms
        for path, cpt, nt, ch, pf, th in itertools.product((2, 3), (4, 8), (32, 64), (1, 2, 4),
                                                            (1, 2), tile_hs):
            if cpt == 8 and radius < 4:
                continue
            out.append({"tile_w": nt * cpt, "tile_h": th, "chunk_rows": ch, "prefetch": pf,
                        "cols_per_thread": cpt, "path": path})
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
               tile_hs=(0,), record: bool = True, verbose: bool = False, cands=None,
               verify=None) -> dict:
    """Search the candidates (`cands`, default `candidates(radius, levels,
    tile_hs)`) on one image (a seeded camera-like image unless `src` is
    given); every candidate must write the same bytes as the first, and
    `verify(cfg, dst)`, if given, is called with each candidate's output.
    Returns {"config", "ms", "results"}."""
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
        for cfg in (candidates(radius, levels, tile_hs) if cands is None else cands):
            try:
                op.set_config(cfg)
            except B.OilPaintError as e:
                if e.status == B.OP_E_UNSUPPORTED:
                    continue
                raise
            ms = _time_filter(op, src, dst, reps)
            if op.sync_status() != B.OP_OK:
                raise B.OilPaintError(f"device error under {cfg}")
            if verify is not None:
                verify(cfg, dst)
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


def save_table(entries: dict, path: str, device_name: str, batch_entries: dict | None = None
               ) -> None:
    table = {"device": device_name, "entries": entries}
    if batch_entries:
        table["batch_entries"] = batch_entries
    with open(path, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)


def batch_candidates() -> list[dict]:
    """Persistent-kernel configurations tried for one batch group: threads
    per CTA x output columns per thread x halo chunk height (one chunk in
    flight)."""
    return [{"tile_w": nt * cpt, "tile_h": 0, "chunk_rows": ch, "prefetch": 1,
             "cols_per_thread": cpt, "path": 0}
            for nt, cpt, ch in itertools.product((32, 64, 128), (1, 2, 4), (1, 2, 4))]


def tune_batch(images: list[dict], max_radius: int, max_levels: int, reps: int = 7,
               rounds: int = 1, verbose: bool = False, cands=None) -> dict:
    """Tune the configuration of each group of a batch created for
    (max_radius, max_levels) on `images` (dicts with src, w, h, stride, bpp,
    r, L; CUDA uint8 sources): coordinate descent over the groups, each
    candidate timed as the median of `reps` graph replays and required to
    write the same bytes as the first.  Records the winners in the library's
    batch table; returns {"max_radius,max_levels": {"config", "ms"}} per group
    and the batch time under the winners."""
    from .filter import Batch

    pix = Batch.padded_pixels([(im["w"], im["h"]) for im in images])
    stream = torch.cuda.Stream()
    outs = [torch.empty_like(im["src"]) for im in images]
    descs = [(im["src"], o, im["w"], im["h"], im["stride"], im["bpp"], im["r"], im["L"])
             for im, o in zip(images, outs)]
    torch.cuda.synchronize()

    def time_batch():
        b = Batch(len(images), pix + 4096, max_radius, max_levels)
        try:
            b.set(descs, stream)
            b.capture(stream)
            for _ in range(2):
                b.launch_graph(stream)
            evs = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(reps)]
            for e0, e1 in evs:
                e0.record(stream)
                b.launch_graph(stream)
                e1.record(stream)
            if b.sync_status(stream) != B.OP_OK:
                raise B.OilPaintError("device error in the batch")
            groups = b.groups()
        finally:
            b.close()
        return statistics.median(e0.elapsed_time(e1) for e0, e1 in evs), groups

    base_ms, groups = time_batch()
    ref = [o.clone() for o in outs]
    keys = [(g["max_radius"], g["max_levels"]) for g in groups]
    best = {k: dict(g["config"]) for k, g in zip(keys, groups)}
    best_ms = base_ms
    for _ in range(rounds):
        for k in keys:
            for cfg in (batch_candidates() if cands is None else cands):
                B.check(B.op_batch_tune_table_set(k[0], k[1], B.op_config_t.make(**cfg)),
                        "op_batch_tune_table_set")
                try:
                    ms, got = time_batch()
                except B.OilPaintError as e:
                    if e.status == B.OP_E_UNSUPPORTED:
                        continue
                    raise
                # a candidate that does not fit the group falls back: skip it
                gcfg = got[keys.index(k)]["config"]
                if any(gcfg[f] != cfg[f] for f in ("tile_w", "chunk_rows", "cols_per_thread",
                                                    "path")):
                    continue
                if not all(torch.equal(a, c) for a, c in zip(ref, outs)):
                    raise B.OilPaintError(f"batch config {cfg} for group {k} changed the output")
                if verbose:
                    print(f"group {k} {cfg} {ms:.4f} ms")
                if ms < best_ms:
                    best_ms, best[k] = ms, dict(cfg)
            B.check(B.op_batch_tune_table_set(k[0], k[1], B.op_config_t.make(**best[k])),
                    "op_batch_tune_table_set")
    return {"groups": {f"{k[0]},{k[1]}": {"config": best[k]} for k in keys},
            "ms": best_ms, "ms_untuned": base_ms}


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
