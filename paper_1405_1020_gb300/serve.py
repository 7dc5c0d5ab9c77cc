"""Continuous-batching server for the oil-paint filter.

Requests (one image each, of any size, radius and level count) arrive from a
client thread with Poisson inter-arrival times.  Their pixels are already on
the device: each request is a strided crop of a device-resident pool of
camera-like images, so no host copy sits on the request path.

The serving loop, every time it wakes:
  1. takes the requests that have arrived since the last pass;
  2. admits waiting requests in arrival order while the bytes they will hold
     on the device (output image + packed-word workspace) fit under the HBM
     cap (40 GB by default) and the device's free memory; a request that can
     never fit is refused with an error instead of waiting forever;
  3. whenever one of its streams is idle, forms a round from the admitted
     requests (up to max_round_images, max_round_mpix) and launches it: the
     round's descriptors go to that stream's batch object (op_batch_set) and
     its captured CUDA graph (the persistent kernel over all tiles of all the
     round's images) is replayed;
  4. retires finished rounds (CUDA event per round), stamping each request's
     completion time and releasing its reservation.
Requests that arrive while rounds run are admitted as memory frees up and go
into the next round on whichever stream is free, so work from different
rounds overlaps on the device (two streams, two batch objects).

Latency = completion (the round's CUDA event, placed on the host clock
through a reference event) minus arrival (when the client released it).
"""
from __future__ import annotations

import collections
import math
import queue
import statistics
import threading
import time
from dataclasses import dataclass, field

from . import synth

OUT_BPP = 3


def padded_pixels(w: int, h: int) -> int:
    return ((w + 3) // 4 * 4) * h


def request_bytes(w: int, h: int) -> int:
    """Device bytes a request holds while admitted: its output image and its
    share of the packed-word workspace."""
    return w * h * OUT_BPP + 4 * padded_pixels(w, h)


@dataclass
class Ticket:
    """A request inside the server."""
    req: synth.Request
    rid: int
    t_arrival: float = 0.0      # host clock (s) when the client released it
    t_done: float | None = None
    out: object = None          # device output tensor while in flight
    round_id: int | None = None
    error: str | None = None


class Admission:
    """Host-side admission and round forming; no device calls, so it can be
    tested on CPU.  `free_bytes` is a callable returning the device's free
    memory (or None to ignore it)."""

    def __init__(self, cap_bytes: int, max_round_images: int, max_round_pixels: int,
                 free_bytes=None, headroom: int = 512 << 20):
        self.cap = cap_bytes
        self.max_images = max_round_images
        self.max_pixels = max_round_pixels
        self.free_bytes = free_bytes
        self.headroom = headroom
        self.reserved = 0
        self.peak_reserved = 0
        self.waiting: collections.deque[Ticket] = collections.deque()
        self.admitted: collections.deque[Ticket] = collections.deque()
        self.refused: list[Ticket] = []

    def arrive(self, t: Ticket) -> None:
        need = request_bytes(t.req.width, t.req.height)
        if need > self.cap or padded_pixels(t.req.width, t.req.height) > self.max_pixels:
            t.error = "request larger than the HBM cap or the round capacity"
            self.refused.append(t)
            return
        self.waiting.append(t)

    def admit(self) -> list[Ticket]:
        """Admit waiting requests in order while they fit; returns them."""
        out = []
        free = self.free_bytes() if self.free_bytes else None
        while self.waiting:
            t = self.waiting[0]
            need = request_bytes(t.req.width, t.req.height)
            if self.reserved + need > self.cap:
                break
            if free is not None and need + self.headroom > free:
                break
            self.waiting.popleft()
            self.reserved += need
            if free is not None:
                free -= need
            self.peak_reserved = max(self.peak_reserved, self.reserved)
            self.admitted.append(t)
            out.append(t)
        return out

    def next_round(self) -> list[Ticket]:
        """Pop the next round from the admitted requests (arrival order)."""
        rnd, pix = [], 0
        while self.admitted and len(rnd) < self.max_images:
            t = self.admitted[0]
            p = padded_pixels(t.req.width, t.req.height)
            if rnd and pix + p > self.max_pixels:
                break
            self.admitted.popleft()
            rnd.append(t)
            pix += p
        return rnd

    def release(self, t: Ticket) -> None:
        self.reserved -= request_bytes(t.req.width, t.req.height)


@dataclass
class _Round:
    rid: int
    tickets: list
    slot: int
    start: object  # CUDA event recorded on the round's stream before its work
    done: object   # CUDA event recorded after it


def overlapping_rounds(spans) -> int:
    """How many rounds ran on the device while a round of another stream was
    also running: spans are (slot, images, start_ms, done_ms) in one device
    time base; two rounds overlap when each started before the other ended."""
    n = 0
    for i, (si, _, ai, bi) in enumerate(spans):
        if any(sj != si and aj < bi and ai < bj
               for j, (sj, _, aj, bj) in enumerate(spans) if j != i):
            n += 1
    return n


@dataclass
class SessionStats:
    offered_mpix_s: float
    duration_s: float
    requests: int
    completed: int
    refused: int
    rounds: int
    mean_round_images: float
    max_round_images: int
    overlapping_rounds: int
    achieved_mpix_s: float
    p50_ms: float
    p99_ms: float
    mean_ms: float
    peak_reserved_gb: float
    samples: list = field(default_factory=list)

    def as_dict(self) -> dict:
        d = dict(self.__dict__)
        d.pop("samples")
        return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in d.items()}


class OilPaintServer:
    """Owns the pool, two streams and one batch object (with its captured
    graph) per stream."""

    def __init__(self, pool, max_radius: int = 20, max_levels: int = 20,
                 max_round_images: int = 64, max_round_mpix: float = 100.0,
                 hbm_cap_bytes: int = 40 * 10**9, nstreams: int = 2, config=None):
        import torch

        from .filter import Batch

        self.torch = torch
        self.pool = pool  # list of (H, W*3) uint8 device tensors
        self.max_radius = max_radius
        self.max_levels = max_levels
        self.max_images = max_round_images
        self.max_pixels = int(max_round_mpix * 1e6)
        self.cap = hbm_cap_bytes
        self.streams = [torch.cuda.Stream() for _ in range(nstreams)]
        self.batches = [Batch(max_round_images, self.max_pixels, max_radius, max_levels,
                              config=config) for _ in range(nstreams)]
        self.captured = [False] * nstreams

    def _descs(self, tickets):
        torch = self.torch
        descs = []
        for t in tickets:
            q = t.req
            img = self.pool[q.pool_index]
            pstride = img.shape[1]
            src = img.view(-1)[q.y0 * pstride + q.x0 * OUT_BPP:]
            t.out = torch.empty(q.width * q.height * OUT_BPP, dtype=torch.uint8,
                                device=img.device)
            descs.append((src, t.out, q.width, q.height, pstride, OUT_BPP, q.radius, q.levels,
                          0, q.width * OUT_BPP))
        return descs

    def serve(self, requests, sample_every: int = 0, idle_sleep_s: float = 50e-6) -> tuple:
        """Serves `requests` (sorted by t_arrival, seconds from the start) as
        they arrive.  Returns (tickets, stats dict pieces)."""
        torch = self.torch
        adm = Admission(self.cap, self.max_images, self.max_pixels,
                        free_bytes=lambda: torch.cuda.mem_get_info()[0])
        inbox: queue.Queue = queue.Queue()
        tickets = [Ticket(req=r, rid=i) for i, r in enumerate(requests)]
        # reference event: GPU timestamps -> host clock
        ref = torch.cuda.Event(enable_timing=True)
        ref.record(self.streams[0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()

        def client():
            for t in tickets:
                delay = t0 + t.req.t_arrival - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                t.t_arrival = time.perf_counter()
                inbox.put(t)
            inbox.put(None)

        th = threading.Thread(target=client, daemon=True)
        th.start()
        client_done = False
        pending: list = []  # an arrival taken from the inbox while idle
        in_flight: dict[int, _Round] = {}
        rounds = 0
        round_sizes = []
        spans = []  # (stream slot, images, start ms, done ms) per finished round
        while not (client_done and not adm.waiting and not adm.admitted and not in_flight):
            busy = False
            while True:
                try:
                    t = pending.pop() if pending else inbox.get_nowait()
                except queue.Empty:
                    break
                if t is None:
                    client_done = True
                else:
                    adm.arrive(t)
                busy = True
            if adm.waiting:
                busy |= bool(adm.admit())
            for slot, stream in enumerate(self.streams):
                if slot in in_flight or not adm.admitted:
                    continue
                rnd = adm.next_round()
                with torch.cuda.stream(stream):
                    start = torch.cuda.Event(enable_timing=True)
                    start.record(stream)
                    descs = self._descs(rnd)
                    b = self.batches[slot]
                    b.set(descs, stream)
                    if not self.captured[slot]:
                        b.capture(stream)
                        self.captured[slot] = True
                    b.launch_graph(stream)
                    done = torch.cuda.Event(enable_timing=True)
                    done.record(stream)
                for t in rnd:
                    t.round_id = rounds
                in_flight[slot] = _Round(rounds, rnd, slot, start, done)
                rounds += 1
                round_sizes.append(len(rnd))
                busy = True
            for slot in list(in_flight):
                rd = in_flight[slot]
                if rd.done.query():
                    done_ms = ref.elapsed_time(rd.done)
                    spans.append((slot, len(rd.tickets), ref.elapsed_time(rd.start), done_ms))
                    t_done = t0 + done_ms / 1e3
                    for t in rd.tickets:
                        t.t_done = t_done
                        adm.release(t)
                        if not (sample_every and t.rid % sample_every == 0):
                            t.out = None  # output delivered; memory returns to the pool
                    del in_flight[slot]
                    busy = True
            if not busy and not client_done:
                # idle: block on the inbox (woken at once by an arrival) for at
                # most idle_sleep_s, then poll the rounds in flight again
                try:
                    pending.append(inbox.get(timeout=idle_sleep_s))
                except queue.Empty:
                    pass
            elif not busy:
                time.sleep(idle_sleep_s)
        t_end = time.perf_counter()
        th.join()
        for b, s in zip(self.batches, self.streams):
            st = b.sync_status(s)
            if st != 0:
                raise RuntimeError(f"device error status {st} in a served round")
        info = {"t0": t0, "t_end": t_end, "rounds": rounds, "round_sizes": round_sizes,
                "round_spans": spans, "refused": len(adm.refused),
                "peak_reserved": adm.peak_reserved}
        return tickets, info

    def close(self):
        for b in self.batches:
            b.close()


def summarize(tickets, info, offered_mpix_s: float, warmup_s: float) -> SessionStats:
    done = [t for t in tickets if t.t_done is not None and t.req.t_arrival >= warmup_s]
    lat = sorted((t.t_done - t.t_arrival) * 1e3 for t in done)
    px = sum(t.req.width * t.req.height for t in done)
    if done:
        span = max(t.t_done for t in done) - min(t.t_arrival for t in done)
    else:
        span = 0.0

    def pct(p):
        if not lat:
            return float("nan")
        k = min(len(lat) - 1, max(0, int(round(p / 100.0 * (len(lat) - 1)))))
        return lat[k]

    return SessionStats(
        offered_mpix_s=offered_mpix_s, duration_s=info["t_end"] - info["t0"],
        requests=len(tickets), completed=len(done), refused=info["refused"],
        rounds=info["rounds"],
        mean_round_images=statistics.mean(info["round_sizes"]) if info["round_sizes"] else 0.0,
        max_round_images=max(info["round_sizes"], default=0),
        overlapping_rounds=overlapping_rounds(info.get("round_spans", [])),
        achieved_mpix_s=px / span / 1e6 if span > 0 else 0.0,
        p50_ms=pct(50), p99_ms=pct(99), mean_ms=statistics.mean(lat) if lat else float("nan"),
        peak_reserved_gb=info["peak_reserved"] / 1e9)


POOL_SHAPE = (4400, 6600)  # H, W: holds the largest (24 MP) requests in either aspect


def make_pool(seed: int = 41):
    import torch
    img = synth.camera_like(POOL_SHAPE[0], POOL_SHAPE[1], seed=seed)
    return [torch.from_numpy(img.reshape(POOL_SHAPE[0], -1)).cuda()]


def check_samples(server: OilPaintServer, tickets) -> int:
    """Re-runs every sampled request alone through op_run; returns how many
    were compared (raises if one differs)."""
    torch = server.torch
    from .filter import OilPaint
    n = 0
    for t in tickets:
        if t.out is None:
            continue
        q = t.req
        img = server.pool[q.pool_index]
        crop = img[q.y0:q.y0 + q.height, q.x0 * OUT_BPP:(q.x0 + q.width) * OUT_BPP].contiguous()
        alone = torch.empty(q.width * q.height * OUT_BPP, dtype=torch.uint8, device=img.device)
        op = OilPaint(q.width, q.height, q.radius, q.levels, bpp=OUT_BPP)
        op.run(crop.view(-1), alone)
        if op.sync_status() != 0:
            raise RuntimeError("device error in a solo re-run")
        op.close()
        if not torch.equal(alone, t.out):
            raise RuntimeError(f"request {t.rid} differs when run alone")
        n += 1
    return n


# Offered load above what the server could take one request at a time: a
# 4.36 MP mean request alone takes about 0.35 ms end to end (about
# 12,000 Mpix/s), so at 20,000 Mpix/s requests queue up and only rounds of
# several requests, overlapping on two streams, keep up.
OVERLOAD_MPIX_S = 20000.0


def bench_loads(seconds: float = 60.0, warmup_s: float = 1.0, loads=(50.0, 200.0, 800.0),
                overload_mpix_s: float | None = OVERLOAD_MPIX_S, overload_seconds: float = 10.0,
                seed: int = 4, sample_every: int = 100) -> dict:
    """Serves Poisson traffic at each offered load (Mpix/s) for `seconds` after
    `warmup_s`, then at `overload_mpix_s` for `overload_seconds`; returns p50/p99
    latency, achieved Mpix/s and the rounds' sizes and overlap per load.  Every
    `sample_every`-th request is re-run alone and must give the same bytes."""
    pool = make_pool()
    server = OilPaintServer(pool)
    mean_px = (24e6 - 0.1e6) / math.log(24e6 / 0.1e6)  # mean of log-uniform 0.1..24 MP
    out = {"workload": "Poisson single-image requests, 0.1-24 MP log-uniform, r uniform 1..20, "
                       "L=20, RGB crops of a device-resident camera-like pool",
           "hbm_cap_gb": 40, "seconds_per_load": seconds, "warmup_s": warmup_s, "loads": []}
    plan = [(load, seconds, "configured") for load in loads]
    if overload_mpix_s:
        plan.append((overload_mpix_s, overload_seconds, "above single-request capacity"))
    try:
        for k, (load, secs, kind) in enumerate(plan):
            rate = load * 1e6 / mean_px
            reqs = synth.poisson_requests(rate, secs + warmup_s, seed=seed + k,
                                          pool_shapes=(POOL_SHAPE,))
            every = sample_every if kind == "configured" else 10 * sample_every
            tickets, info = server.serve(reqs, sample_every=every)
            st = summarize(tickets, info, load, warmup_s)
            d = {"kind": kind, **st.as_dict()}
            d["seconds"] = secs
            d["rate_req_s"] = round(rate, 2)
            d["resampled_identical"] = check_samples(server, tickets)
            out["loads"].append(d)
    finally:
        server.close()
    return out
