#!/usr/bin/env python3
"""Benchmark of the GB300 oil-paint filter: Mpix/s on the 12 MP workload.

Workload (one "step" = the whole hot path on one image): a 4000x3000
camera-like synthetic image (seed 2) stored as RGBA rows of 16000 bytes,
radius 15 (31x31 window), L = 20 levels: the pack prepass plus the tiled
sliding-histogram filter, launched through the C ABI (op_run) on inputs
already resident in HBM.  Between timed steps a 512 MiB buffer is written to
flush the 129 MB L2.

One JSON line is printed (rank 0).  Besides the headline it carries
  roofline      the filter kernel against the integer-ALU peak,
  e2e           the same metric through op_run_host (host buffers, copies
                included),
  cpu_baseline  the CPU oracle on a bounded row band of the same image,
  batched       the 64-image mixed batch, one persistent launch (CUDA graph)
                vs one plain op_run per image,
  served        the continuous-batching server at 50/200/800 Mpix/s offered
                (60 s per load), then 10 s at 20,000 Mpix/s, above what it could
                serve one request at a time; rounds' sizes and overlap reported,
  clocks        SM clocks and throttle reasons sampled during the timed region.

--impl reference runs the CPU oracle (the only other implementation) on the
same workload, a bounded row band per step.

Under torchrun (--gpus N > 1) every rank runs an independent replica of the
workload on its own GPU (the filter needs no exchange between images); the
reported time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W, H, BPP, STRIDE, RADIUS, LEVELS, SEED = 4000, 3000, 4, 16000, 15, 20, 2
WORKLOAD = "camera-like 4000x3000 RGBA-stride r=15 L=20"
METRIC = "oil-paint Mpix/s at 12MP r=15 L=20"
# Integer-ALU lanes per SM used for the roofline peak (SMs x lanes x max clock).
INT_LANES_PER_SM = 128


def ops_per_pixel(r: int, L: int) -> int:
    """Algorithmic integer operations per output pixel of the sliding
    histogram: 2(2r+1) bin updates of 4 adds each (count, R, G, B sums), an
    L-way argmax, and ~11 for the three divisions and the store."""
    return 16 * r + L + 11


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def reduce_max(x: float) -> float:
    """Maximum of x over the ranks of the default process group (x itself
    when there is none); the tensor lives where the backend wants it."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks/throttle sampling while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, log_path: str | None = None):
        self.gpu = gpu_index
        self.log_path = log_path
        self.proc = None
        self.tmp = None

    def __enter__(self):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.tmp.flush()

    def summary(self):
        self.tmp.seek(0)
        text = self.tmp.read()
        if self.log_path:
            with open(self.log_path, "w") as f:
                f.write(text)
        os.unlink(self.tmp.name)
        rows = [r for r in csv.reader(io.StringIO(text)) if len(r) >= 9]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ workloads

def make_image():
    from paper_1405_1020_gb300 import synth
    img = synth.camera_like(H, W, seed=SEED)
    buf, stride = synth.to_strided(img, bpp=BPP, stride=STRIDE)
    return buf


def cpu_baseline(buf, target_s: float = 10.0):
    """The oracle, as it stands, on a band of rows of the same image."""
    import oracle
    cores = oracle.num_cpus()
    y0 = 0
    probe = 32
    t = time.perf_counter()
    oracle.oilpaint_rows(buf, W, H, STRIDE, BPP, RADIUS, LEVELS, y0, y0 + probe)
    dt = time.perf_counter() - t
    rows = int(max(probe, min(H - y0, round(probe * target_s / max(dt, 1e-6)))))
    t = time.perf_counter()
    oracle.oilpaint_rows(buf, W, H, STRIDE, BPP, RADIUS, LEVELS, y0, y0 + rows)
    dt = time.perf_counter() - t
    return {"value": round(W * rows / dt / 1e6, 4), "unit": "Mpix/s", "cores": cores,
            "kind": "oracle",
            "sample": f"rows {y0}..{y0 + rows - 1} ({W * rows / 1e6:.3f} Mpix) of the "
                      f"{WORKLOAD} image, C oracle on {cores} threads, {dt:.2f} s"}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import oracle
    buf = make_image()
    cores = oracle.num_cpus()
    rows = args.ref_rows
    y0 = H // 2
    for _ in range(args.warmup):
        oracle.oilpaint_rows(buf, W, H, STRIDE, BPP, RADIUS, LEVELS, y0, y0 + rows)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.oilpaint_rows(buf, W, H, STRIDE, BPP, RADIUS, LEVELS, y0, y0 + rows)
        times.append(time.perf_counter() - t)
    ms = 1e3 * statistics.mean(times)
    value = W * rows / (ms / 1e3) / 1e6
    sample = f"rows {y0}..{y0 + rows - 1} ({W * rows / 1e6:.3f} Mpix) per step, C oracle"
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "Mpix/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "width": W, "height": H, "bpp": BPP, "radius": RADIUS,
                   "levels": LEVELS, "sample_rows": rows},
        "cpu_baseline": {"value": round(value, 4), "unit": "Mpix/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    from paper_1405_1020_gb300 import binding as B
    from paper_1405_1020_gb300.filter import OilPaint

    rank, world, local = dist_info()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    __graft_entry__.build()

    buf = make_image()
    src = torch.from_numpy(buf).cuda()
    dst = torch.zeros_like(src)
    cfg = json.loads(args.config) if args.config else None
    tuned = None
    if args.autotune and cfg is None:
        from paper_1405_1020_gb300 import autotune
        tuned = autotune.tune_image(W, H, BPP, STRIDE, RADIUS, LEVELS, src=src)
        cfg = tuned["config"]
    op = OilPaint(W, H, RADIUS, LEVELS, bpp=BPP, stride=STRIDE, config=cfg)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        op.run(src, dst)
    torch.cuda.synchronize()
    if op.sync_status() != B.OP_OK:
        raise RuntimeError("device error during warm-up")

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    for e in ev:  # create the CUDA events before handing one to the library
        e[1].record(stream)
    torch.cuda.synchronize()

    sampler = ClockSampler(local, os.path.join(args.out_dir, f"clocks_rank{rank}.csv")
                           if args.out_dir else None)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with sampler:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            B.check(B.op_set_profile_event(op.handle, ev[k][1].cuda_event), "profile event")
            ev[k][0].record(stream)
            op.run(src, dst)
            ev[k][2].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    B.op_set_profile_event(op.handle, None)
    if world > 1:
        dist.barrier()
    if op.sync_status() != B.OP_OK:
        raise RuntimeError("device error during the timed steps")
    clocks = sampler.summary()

    step_ms = [e[0].elapsed_time(e[2]) for e in ev]
    pack_ms = [e[0].elapsed_time(e[1]) for e in ev]
    filt_ms = [e[1].elapsed_time(e[2]) for e in ev]
    ms = reduce_max(statistics.mean(step_ms))
    value = world * W * H / (ms / 1e3) / 1e6

    # roofline of the dominant kernel (the filter): integer-ALU bound
    peaks = read_peaks() or {}
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak_tops = sms * INT_LANES_PER_SM * sm_max * 1e6 / 1e12
    f_ms = statistics.mean(filt_ms)
    ach_tops = ops_per_pixel(RADIUS, LEVELS) * W * H / (f_ms / 1e3) / 1e12
    traffic = None
    pipe = None
    tpath = os.path.join(ROOT, "profiles", "filter_traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tr = json.load(f)
        if tr.get("workload") == WORKLOAD and tr.get("kernel_source_hash") == _kernel_hash():
            traffic = tr.get("bytes_per_launch")
            if tr.get("shared_pipe_pct") is not None:
                # the pipe that bounds the kernel in the same capture
                pipe = {"pipe": "shared memory (l1tex)",
                        "frac": round(tr["shared_pipe_pct"] / 100.0, 4),
                        "issue_active": round(tr.get("issue_active_pct", 0.0) / 100.0, 4),
                        "source": "ncu, " + tr.get("summary", "")}
    launch = op.config()
    if launch.get("path", 0) == 1:
        kernel = "tile_cols_kernel"
    elif launch.get("path", 0) >= 2 or launch["cols_per_thread"] == 8:
        kernel = "tile_deltak_kernel"
    elif launch["cols_per_thread"] > 1 and LEVELS <= 32:
        kernel = "tile_delta_kernel"
    else:
        kernel = "tile_plain_kernel"
    roofline = {"bound": "alu", "achieved": round(ach_tops, 3), "peak": round(peak_tops, 3),
                "unit": "Tops/s", "frac": round(ach_tops / peak_tops, 4), "traffic": traffic,
                "kernel": kernel, "kernel_ms": round(f_ms, 4),
                "pack_ms": round(statistics.mean(pack_ms), 4),
                "ops_per_pixel": ops_per_pixel(RADIUS, LEVELS),
                "peak_source": f"{sms} SMs x {INT_LANES_PER_SM} int lanes x {sm_max:.0f} MHz "
                               "(lanes measured: profiles/alu_peak_probe.md)",
                "bounding_pipe": pipe}

    # end to end through the host-buffer entry points: every step copies its
    # input from pinned host memory and its result back.  op_run_host_async
    # lets consecutive steps overlap (copy in / filter / copy out on the op's
    # own streams); op_run_host is the synchronous, one-at-a-time form.
    h_in = torch.from_numpy(buf).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    e2e_stream = torch.cuda.Stream()
    n_e2e = max(10, args.steps)
    for _ in range(3):
        op.run_host_async(h_in, h_out, e2e_stream)
    e2e_stream.synchronize()
    if world > 1:
        dist.barrier()
    t = time.perf_counter()
    for _ in range(n_e2e):
        op.run_host_async(h_in, h_out, e2e_stream)
    e2e_stream.synchronize()
    e2e_s = reduce_max((time.perf_counter() - t) / n_e2e)
    if op.sync_status(e2e_stream) != B.OP_OK:
        raise RuntimeError("device error in the host-buffer steps")
    sync_times = []
    for _ in range(max(3, args.steps // 4)):
        t = time.perf_counter()
        op.run_host(h_in, h_out)
        sync_times.append(time.perf_counter() - t)
    sync_s = reduce_max(statistics.mean(sync_times))
    e2e = {"value": round(world * W * H / e2e_s / 1e6, 3), "unit": "Mpix/s",
           "h2d_bytes_per_step": H * STRIDE, "d2h_bytes_per_step": H * W * BPP,
           "steps": n_e2e, "ms_per_step": round(e2e_s * 1e3, 4),
           "api": "op_run_host_async (consecutive steps overlap copies and filter)",
           "sync_value": round(world * W * H / sync_s / 1e6, 3),
           "sync_api": "op_run_host (one step at a time)"}
    if not np.array_equal(h_out.numpy(), dst.cpu().numpy()):
        raise RuntimeError("op_run_host output differs from op_run output")

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mpix/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "width": W, "height": H, "bpp": BPP, "stride": STRIDE,
                   "radius": RADIUS, "levels": LEVELS, "seed": SEED,
                   "launch": op.config(), "autotuned": tuned is not None,
                   "l2": "flushed between steps (512 MiB write)"},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "wall_s_timed_region": round(t_wall, 4),
    }
    # The batch, JPEG and served measurements describe one GPU: they run in
    # the single-GPU job only, so that a multi-GPU run holds its GPUs for the
    # headline steps alone.
    if not args.skip_batch and world == 1:
        from paper_1405_1020_gb300 import batchbench
        line["batched"] = batchbench.run(steps=max(3, args.steps // 2), warmup=2)
    if not args.skip_jpeg and world == 1:
        from paper_1405_1020_gb300 import jpegbench
        line["jpeg_pipeline"] = jpegbench.run()
    if args.serve_seconds > 0 and world == 1:
        from paper_1405_1020_gb300 import serve
        line["served"] = serve.bench_loads(seconds=args.serve_seconds,
                                           overload_seconds=args.overload_seconds)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(buf, args.cpu_seconds)
    op.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1405_1020_gb300", "csrc")
    for name in ("oilpaint_device.cuh", "oilpaint_kernels.cu", "oilpaint_deltak.cuh"):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--config", default=None, help="launch config JSON, e.g. '{\"tile_w\": 64}'")
    p.add_argument("--autotune", action="store_true", help="search the launch config first")
    p.add_argument("--skip-batch", action="store_true")
    p.add_argument("--skip-jpeg", action="store_true",
                   help="skip the decode -> filter -> encode timing")
    p.add_argument("--serve-seconds", type=float, default=60.0,
                   help="seconds of served traffic per configured offered load (0 skips "
                        "serving)")
    p.add_argument("--overload-seconds", type=float, default=10.0,
                   help="seconds of served traffic at the load above single-request capacity")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--ref-rows", type=int, default=96, help="rows per reference step")
    p.add_argument("--out-dir", default=None, help="where to keep the clock samples")
    args = p.parse_args(argv)
    if args.warmup < 3:
        p.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
