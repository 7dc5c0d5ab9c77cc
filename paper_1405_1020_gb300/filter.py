"""Torch-facing wrappers over the C ABI.

PyTorch provides device memory (the workspace and the image tensors) and
streams; every step of the filter runs in the library's CUDA kernels.  There
is no CPU path: without the built library every call raises OilPaintError.
"""
from __future__ import annotations

import ctypes
import json
import os
from typing import Iterable, Sequence

import numpy as np
import torch

from . import binding as B

TUNING_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")
_tuned_loaded = False


def load_tuning(path: str = TUNING_TABLE) -> int:
    """Load the autotuner's saved (radius, levels) -> launch-configuration
    table, and its batch-group table keyed by a group's largest radius and
    level count, into the library (once per process unless `path` is given
    explicitly); returns the number of single-image entries."""
    global _tuned_loaded
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        table = json.load(f)
    entries = table.get("entries", {})
    for key, ent in entries.items():
        r, L = (int(v) for v in key.split(","))
        B.check(B.op_tune_table_set(r, L, B.op_config_t.make(**ent["config"])), "tune table")
    for key, ent in table.get("batch_entries", {}).items():
        r, L = (int(v) for v in key.split(","))
        B.check(B.op_batch_tune_table_set(r, L, B.op_config_t.make(**ent["config"])),
                "batch tune table")
    _tuned_loaded = True
    return len(entries)


def _ensure_tuned() -> None:
    if not _tuned_loaded:
        load_tuning()


def _stream_handle(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check_dev_buf(t: torch.Tensor, nbytes: int, name: str) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise B.OilPaintError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.uint8 or not t.is_contiguous():
        raise B.OilPaintError(f"{name} must be a contiguous uint8 tensor")
    if t.numel() < nbytes:
        raise B.OilPaintError(f"{name} holds {t.numel()} bytes, needs {nbytes}")


def _config(cfg) -> B.op_config_t:
    if cfg is None or isinstance(cfg, B.op_config_t):
        return cfg
    d = dict(cfg)
    return B.op_config_t.make(d.get("tile_w", 128), d.get("tile_h", 0), d.get("chunk_rows", 8),
                              d.get("prefetch", 2), d.get("cols_per_thread", 1),
                              d.get("path", 0))


class OilPaint:
    """One image geometry: width x height pixels, `bpp` bytes per pixel, rows
    `stride` bytes apart, radius r, L levels (section 4's filter)."""

    def __init__(self, width: int, height: int, radius: int, levels: int, bpp: int = 3,
                 stride: int | None = None, flags: int = B.OP_LEVEL_PAPER, config=None,
                 device: int | torch.device | None = None):
        self.width, self.height, self.radius, self.levels = width, height, radius, levels
        self.bpp = bpp
        self.stride = stride if stride is not None else width * bpp
        self.flags = flags
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self._h = None
        _ensure_tuned()
        with torch.cuda.device(self.device):
            h = B.op_create_ex(width, height, self.stride, bpp, radius, levels, flags)
            if not h:
                st = B.op_last_error()
                raise B.OilPaintError(f"op_create_ex: {B.status_string(st)}", st)
            self._h = h
            if config is not None:
                B.check(B.op_set_config(h, _config(config)), "op_set_config")
            n = B.op_workspace_size(h)
            self._ws = torch.empty(max(n, 16), dtype=torch.uint8, device=self.device)
            B.check(B.op_set_workspace(h, self._ws.data_ptr(), self._ws.numel()),
                    "op_set_workspace")

    @property
    def nbytes(self) -> int:
        return self.height * self.stride

    @property
    def handle(self):
        return self._h

    def config(self) -> dict:
        c = B.op_config_t()
        B.check(B.op_get_config(self._h, c), "op_get_config")
        return c.as_dict()

    def set_config(self, cfg) -> None:
        B.check(B.op_set_config(self._h, _config(cfg)), "op_set_config")

    def run(self, src: torch.Tensor, dst: torch.Tensor, stream=None) -> None:
        """Asynchronous on `stream` (default: torch's current stream)."""
        _check_dev_buf(src, self.nbytes, "src")
        _check_dev_buf(dst, self.nbytes, "dst")
        B.check(B.op_run(self._h, src.data_ptr(), dst.data_ptr(), _stream_handle(stream)),
                "op_run")

    def __call__(self, src: torch.Tensor, dst: torch.Tensor | None = None, stream=None):
        if dst is None:
            dst = torch.empty_like(src)
        self.run(src, dst, stream)
        return dst

    def _host_ptr(self, a) -> int:
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.uint8 or not a.is_contiguous():
                raise B.OilPaintError("host buffers must be contiguous uint8 CPU tensors")
            if a.numel() < self.nbytes:
                raise B.OilPaintError("host buffer too small")
            return a.data_ptr()
        a = np.asarray(a)
        if a.dtype != np.uint8 or not a.flags["C_CONTIGUOUS"] or a.size < self.nbytes:
            raise B.OilPaintError("host buffers must be contiguous uint8 arrays")
        return a.ctypes.data

    def run_host(self, h_in, h_out, stream=None) -> None:
        """Host buffers in and out (numpy arrays or CPU tensors, ideally pinned);
        synchronous."""
        B.check(B.op_run_host(self._h, self._host_ptr(h_in), self._host_ptr(h_out),
                              _stream_handle(stream)), "op_run_host")

    def run_host_async(self, h_in, h_out, stream=None) -> None:
        """Enqueue the host-buffer filter; consecutive calls overlap one image's
        copies with another's filter.  `stream` waits for the result: keep both
        buffers alive (and pinned) until it is synchronised or sync_status()."""
        B.check(B.op_run_host_async(self._h, self._host_ptr(h_in), self._host_ptr(h_out),
                                    _stream_handle(stream)), "op_run_host_async")

    def sync_status(self, stream=None) -> int:
        return B.op_sync_status(self._h, _stream_handle(stream))

    def close(self) -> None:
        if self._h:
            B.op_destroy(self._h)
            self._h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Many images in one persistent launch (see op_batch_create)."""

    def __init__(self, max_images: int, max_pixels: int, max_radius: int, max_levels: int,
                 config=None, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self._h = None
        _ensure_tuned()
        with torch.cuda.device(self.device):
            h = B.op_batch_create(max_images, max_pixels, max_radius, max_levels, _config(config))
            if not h:
                st = B.op_last_error()
                raise B.OilPaintError(f"op_batch_create: {B.status_string(st)}", st)
            self._h = h
            n = B.op_batch_workspace_size(h)
            self._ws = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
            base = self._ws.data_ptr()
            aligned = (base + 255) // 256 * 256
            self._ws_off = aligned - base
            B.check(B.op_batch_set_workspace(h, aligned, n), "op_batch_set_workspace")
        self._keep: list = []
        self.n = 0

    @staticmethod
    def padded_pixels(images: Iterable[tuple]) -> int:
        """Pixels the batch workspace needs for images given as (w, h, ...)."""
        return sum(((w + 3) // 4 * 4) * h for w, h, *_ in images)

    def set(self, images: Sequence[tuple], stream=None) -> None:
        """images: (src, dst, width, height, stride, bpp, radius, levels[, flags
        [, out_stride]]) with src/dst CUDA uint8 tensors; out_stride is the
        output's row pitch (default: stride)."""
        arr = (B.op_image_t * max(1, len(images)))()
        keep = []
        for i, im in enumerate(images):
            src, dst, w, h, stride, bpp, r, L = im[:8]
            flags = im[8] if len(im) > 8 else B.OP_LEVEL_PAPER
            ostride = im[9] if len(im) > 9 and im[9] else stride
            # a strided crop only needs its last row's pixels after (h-1) pitches
            _check_dev_buf(src, (h - 1) * stride + w * bpp, f"images[{i}].src")
            _check_dev_buf(dst, (h - 1) * ostride + w * bpp, f"images[{i}].dst")
            arr[i] = B.op_image_t(src.data_ptr(), dst.data_ptr(), w, h, stride, bpp, r, L, flags,
                                  ostride)
            keep += [src, dst]
        B.check(B.op_batch_set(self._h, arr, len(images), _stream_handle(stream)), "op_batch_set")
        self._keep = keep
        self.n = len(images)

    def config(self) -> dict:
        c = B.op_config_t()
        B.check(B.op_batch_get_config(self._h, c), "op_batch_get_config")
        return c.as_dict()

    def groups(self) -> list[dict]:
        """Each image group's largest radius and level count and its launch
        configuration."""
        out = []
        for g in range(B.op_batch_group_count(self._h)):
            c, r, L = B.op_config_t(), ctypes.c_int32(), ctypes.c_uint32()
            B.check(B.op_batch_get_group(self._h, g, c, r, L), "op_batch_get_group")
            out.append({"max_radius": r.value, "max_levels": L.value, "config": c.as_dict()})
        return out

    def diagnostics(self) -> list[int]:
        """The timeout diagnostic record of the batch's control block (16
        words: a set flag, then image w, h, tile x0, y0, y1, chunk, chunks,
        global chunk, ring slots, expected parity, chunks issued, barrier
        word lo/hi, r | L << 16, box width | chunk rows << 16)."""
        torch.cuda.synchronize()
        words = self._ws[self._ws_off + 32:self._ws_off + 96].cpu().numpy().view("<u4")
        return [int(v) for v in words]

    def run(self, stream=None) -> None:
        B.check(B.op_batch_run(self._h, _stream_handle(stream)), "op_batch_run")

    def capture(self, stream) -> None:
        """Capture run() into a CUDA graph; `stream` must be a non-default stream."""
        B.check(B.op_batch_capture(self._h, _stream_handle(stream)), "op_batch_capture")

    def launch_graph(self, stream=None) -> None:
        B.check(B.op_batch_launch_graph(self._h, _stream_handle(stream)), "op_batch_launch_graph")

    def sync_status(self, stream=None) -> int:
        return B.op_batch_sync_status(self._h, _stream_handle(stream))

    def close(self) -> None:
        if self._h:
            B.op_batch_destroy(self._h)
            self._h = None
            self._ws = None
            self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

