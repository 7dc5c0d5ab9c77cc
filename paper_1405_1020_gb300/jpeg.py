"""ctypes binding of include/oilpaint_jpeg.h -- the decode -> filter -> encode
pipeline of section 3.2 (Decode, ApplyOilPaintOnBuffer, Encode,
ApplyOilPaintOnFile) with nvJPEG as the codec.

The same-named functions marshal arguments only and return the C status.
``JpegPipeline`` wraps them for torch users: JPEG bytes in and out as Python
``bytes``, device images as uint8 CUDA tensors of ``height x pitch`` bytes
(interleaved R, G, B), errors raised as ``OilPaintError``.

The library is ``liboilpaint_jpeg.so`` next to this file, built by
``__graft_entry__.build()`` when the CUDA toolkit has nvJPEG.  There is no
fallback codec: if the library is missing, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

from . import binding
from .binding import OP_OK, OilPaintError

OP_E_CODEC = -7
OP_E_NOSPACE = -8

OP_JPEG_CSS_444 = 0
OP_JPEG_CSS_422 = 1
OP_JPEG_CSS_420 = 2

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liboilpaint_jpeg.so")

# every symbol include/oilpaint_jpeg.h declares
EXPORTS = (
    "op_jpeg_create", "op_jpeg_last_error", "op_jpeg_info", "op_jpeg_decode",
    "op_jpeg_encode_bound", "op_jpeg_encode", "op_jpeg_filter", "op_jpeg_filter_file",
    "op_jpeg_filter_batch", "op_jpeg_last_timing", "op_jpeg_destroy",
)

OP_JPEG_MAX_BATCH = 64


class op_jpeg_timing_t(ctypes.Structure):
    _fields_ = [("decode_ms", ctypes.c_float), ("filter_ms", ctypes.c_float),
                ("encode_ms", ctypes.c_float)]


_lib = None


def available(path: str = LIB_PATH) -> bool:
    return os.path.exists(path)


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liboilpaint_jpeg.so (once, after liboilpaint.so) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OilPaintError(f"{path} is not built (the CUDA toolkit needs nvJPEG); "
                            "run __graft_entry__.build()")
    binding.load()
    lib = ctypes.CDLL(path)
    u32, i32, sz, ci, vp = ctypes.c_uint32, ctypes.c_int32, ctypes.c_size_t, ctypes.c_int, ctypes.c_void_p
    cp, pu32, psz = ctypes.c_char_p, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_size_t)
    sig = {
        "op_jpeg_create": (vp, [vp]),
        "op_jpeg_last_error": (ci, []),
        "op_jpeg_info": (ci, [vp, cp, sz, pu32, pu32, pu32]),
        "op_jpeg_decode": (ci, [vp, cp, sz, vp, u32, vp]),
        "op_jpeg_encode_bound": (ci, [vp, u32, u32, ci, ci, psz]),
        "op_jpeg_encode": (ci, [vp, vp, u32, u32, u32, ci, ci, vp, sz, psz, vp]),
        "op_jpeg_filter": (ci, [vp, cp, sz, i32, u32, u32, ci, ci, vp, sz, psz, vp, u32, vp]),
        "op_jpeg_filter_file": (ci, [vp, cp, cp, i32, u32, u32, ci, ci, vp]),
        "op_jpeg_filter_batch": (ci, [vp, u32, ctypes.POINTER(vp), psz, i32, u32, u32, ci, ci,
                                      ctypes.POINTER(vp), psz, psz, ctypes.POINTER(ci), vp]),
        "op_jpeg_last_timing": (ci, [vp, ctypes.POINTER(op_jpeg_timing_t)]),
        "op_jpeg_destroy": (ci, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    if status == OP_E_CODEC:
        return "nvJPEG rejected the stream or failed"
    if status == OP_E_NOSPACE:
        return "output buffer too small"
    return binding.status_string(status)


def check(status: int, what: str = "call") -> int:
    if status != OP_OK:
        raise OilPaintError(f"{what} failed: {status_string(status)} ({status})", status)
    return status


# ---- same-named wrappers (argument marshalling only) ----------------------

def op_jpeg_create(stream=None):
    return load().op_jpeg_create(stream)


def op_jpeg_last_error():
    return load().op_jpeg_last_error()


def op_jpeg_info(jp, data: bytes, width, height, components):
    """width / height / components: ctypes.c_uint32 (or None)."""
    ref = lambda x: None if x is None else ctypes.byref(x)  # noqa: E731
    return load().op_jpeg_info(jp, data, len(data), ref(width), ref(height), ref(components))


def op_jpeg_decode(jp, data: bytes, d_rgb, pitch, stream=None):
    return load().op_jpeg_decode(jp, data, len(data), d_rgb, pitch, stream)


def op_jpeg_encode_bound(jp, width, height, quality, sampling, nbytes: ctypes.c_size_t):
    return load().op_jpeg_encode_bound(jp, width, height, quality, sampling, ctypes.byref(nbytes))


def op_jpeg_encode(jp, d_rgb, width, height, pitch, quality, sampling, out, cap,
                   out_bytes: ctypes.c_size_t, stream=None):
    return load().op_jpeg_encode(jp, d_rgb, width, height, pitch, quality, sampling, out, cap,
                                 ctypes.byref(out_bytes), stream)


def op_jpeg_filter(jp, data: bytes, radius, levels, flags, quality, sampling, out, cap,
                   out_bytes: ctypes.c_size_t, d_filtered=None, filtered_pitch=0, stream=None):
    return load().op_jpeg_filter(jp, data, len(data), radius, levels, flags, quality, sampling,
                                 out, cap, ctypes.byref(out_bytes), d_filtered, filtered_pitch,
                                 stream)


def op_jpeg_filter_file(jp, in_path: str, out_path: str, radius, levels, flags, quality,
                        sampling, stream=None):
    return load().op_jpeg_filter_file(jp, os.fsencode(in_path), os.fsencode(out_path), radius,
                                      levels, flags, quality, sampling, stream)


def op_jpeg_filter_batch(jp, datas, radius, levels, flags, quality, sampling, outs, caps,
                         out_bytes, status, stream=None):
    """datas: a sequence of JPEG byte strings (kept alive by the caller);
    outs: a ctypes array of output addresses (c_void_p); caps, out_bytes:
    ctypes arrays of c_size_t; status: a ctypes array of c_int; one entry per
    image."""
    n = len(datas)
    ins = (ctypes.c_void_p * max(n, 1))(
        *[ctypes.cast(ctypes.c_char_p(d), ctypes.c_void_p) for d in datas])
    lens = (ctypes.c_size_t * max(n, 1))(*[len(d) for d in datas])
    return load().op_jpeg_filter_batch(jp, n, ins, lens, radius, levels, flags, quality,
                                       sampling, outs, caps, out_bytes, status, stream)


def op_jpeg_last_timing(jp, t: op_jpeg_timing_t):
    return load().op_jpeg_last_timing(jp, ctypes.byref(t))


def op_jpeg_destroy(jp):
    return load().op_jpeg_destroy(jp)


# ---- torch wrapper ---------------------------------------------------------

def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


class JpegPipeline:
    """One codec context (``op_jpeg_t``) on the current CUDA device.

    ``filter(data, radius, levels)`` is ApplyOilPaintOnFile on bytes: decode,
    filter, encode, returning the encoded bytes (and, with ``keep_rgb=True``,
    the filtered RGB tensor it encoded).  ``decode`` / ``encode`` are the two
    codec halves on their own."""

    def __init__(self, stream=None):
        self._h = op_jpeg_create(_stream_handle(stream))
        if not self._h:
            check(op_jpeg_last_error(), "op_jpeg_create")
        self._out = None          # host output buffer, reused across calls

    def _outbuf(self, cap: int):
        import numpy as np
        if self._out is None or self._out.size < cap:
            self._out = np.empty(cap, dtype=np.uint8)
        return self._out.ctypes.data_as(ctypes.c_void_p)

    def close(self):
        if self._h:
            op_jpeg_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self, data: bytes):
        """(width, height, components) from the JPEG headers."""
        w, h, c = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        check(op_jpeg_info(self._h, data, w, h, c), "op_jpeg_info")
        return w.value, h.value, c.value

    def decode(self, data: bytes, pitch: int | None = None, stream=None):
        """Decoded image as a uint8 CUDA tensor of shape (height, pitch)."""
        import torch
        w, h, _ = self.info(data)
        pitch = 3 * w if pitch is None else pitch
        out = torch.empty((h, pitch), dtype=torch.uint8, device="cuda")
        check(op_jpeg_decode(self._h, data, out.data_ptr(), pitch, _stream_handle(stream)),
              "op_jpeg_decode")
        return out

    def encode_bound(self, width: int, height: int, quality: int = 90,
                     sampling: int = OP_JPEG_CSS_420) -> int:
        n = ctypes.c_size_t()
        check(op_jpeg_encode_bound(self._h, width, height, quality, sampling, n),
              "op_jpeg_encode_bound")
        return n.value

    def encode(self, rgb, width: int, height: int, pitch: int | None = None, quality: int = 90,
               sampling: int = OP_JPEG_CSS_420, stream=None) -> bytes:
        """Encode a uint8 CUDA tensor of height rows of `pitch` bytes."""
        pitch = 3 * width if pitch is None else pitch
        cap = self.encode_bound(width, height, quality, sampling)
        buf = self._outbuf(cap)
        n = ctypes.c_size_t()
        check(op_jpeg_encode(self._h, rgb.data_ptr(), width, height, pitch, quality, sampling,
                             buf, cap, n, _stream_handle(stream)), "op_jpeg_encode")
        return self._out[:n.value].tobytes()

    def filter(self, data: bytes, radius: int, levels: int, flags: int = 0, quality: int = 90,
               sampling: int = OP_JPEG_CSS_420, keep_rgb: bool = False, stream=None):
        import torch
        w, h, _ = self.info(data)
        cap = self.encode_bound(w, h, quality, sampling)
        buf = self._outbuf(cap)
        n = ctypes.c_size_t()
        rgb = torch.empty((h, 3 * w), dtype=torch.uint8, device="cuda") if keep_rgb else None
        check(op_jpeg_filter(self._h, data, radius, levels, flags, quality, sampling, buf, cap, n,
                             None if rgb is None else rgb.data_ptr(), 3 * w if keep_rgb else 0,
                             _stream_handle(stream)), "op_jpeg_filter")
        out = self._out[:n.value].tobytes()
        return (out, rgb) if keep_rgb else out

    def filter_batch(self, datas, radius: int, levels: int, flags: int = 0, quality: int = 90,
                     sampling: int = OP_JPEG_CSS_420, stream=None) -> list:
        """filter() over a list of JPEG byte strings in one op_jpeg_filter_batch
        call (one batched decode on the GPU's JPEG engines where the streams
        allow it); the encoded outputs in input order.  Raises OilPaintError
        for the first image that failed."""
        import numpy as np
        datas = [bytes(d) for d in datas]
        n = len(datas)
        if n == 0:
            return []
        caps = []
        for d in datas:
            try:
                w, h, _ = self.info(d)
                caps.append(self.encode_bound(w, h, quality, sampling))
            except OilPaintError:
                caps.append(0)        # the call reports this image's status
        buf = np.empty(max(1, sum(caps)), dtype=np.uint8)
        offs = np.concatenate(([0], np.cumsum(caps)[:-1])).astype(np.int64)
        base = buf.ctypes.data
        outs = (ctypes.c_void_p * n)(*[base + int(o) for o in offs])
        capa = (ctypes.c_size_t * n)(*caps)
        got = (ctypes.c_size_t * n)()
        status = (ctypes.c_int * n)()
        st = op_jpeg_filter_batch(self._h, datas, radius, levels, flags, quality, sampling, outs,
                                  capa, got, status, _stream_handle(stream))
        if st != OP_OK:
            bad = next((i for i in range(n) if status[i] != OP_OK), None)
            what = "op_jpeg_filter_batch" if bad is None else f"op_jpeg_filter_batch (image {bad})"
            check(st, what)
        return [buf[int(o):int(o) + got[i]].tobytes() for i, o in enumerate(offs)]

    def filter_file(self, in_path: str, out_path: str, radius: int, levels: int, flags: int = 0,
                    quality: int = 90, sampling: int = OP_JPEG_CSS_420, stream=None):
        check(op_jpeg_filter_file(self._h, in_path, out_path, radius, levels, flags, quality,
                                  sampling, _stream_handle(stream)), "op_jpeg_filter_file")

    def last_timing(self) -> dict:
        t = op_jpeg_timing_t()
        check(op_jpeg_last_timing(self._h, t), "op_jpeg_last_timing")
        return {"decode_ms": t.decode_ms, "filter_ms": t.filter_ms, "encode_ms": t.encode_ms}



class JpegPool:
    """`workers` host threads, each with its own codec context (JpegPipeline)
    on its own CUDA stream, kept across calls.  With batch = 1 each thread
    takes one image at a time (JpegPipeline.filter): one image's Huffman
    decoding on the host (nvJPEG's simple decode call, which holds a host core
    for most of an image's time) then overlaps other images' decoding and
    their filtering and encoding on the GPU.  With batch > 1 each thread
    takes `batch` images at a time (JpegPipeline.filter_batch), decoded
    together on the GPU's JPEG engines where the streams allow it.  ctypes
    releases the interpreter lock during the library calls."""

    def __init__(self, workers: int = 4, batch: int = 8):
        if not 1 <= batch <= OP_JPEG_MAX_BATCH:
            raise ValueError(f"batch must be 1..{OP_JPEG_MAX_BATCH}")
        self._batch = batch
        import threading
        from concurrent.futures import ThreadPoolExecutor

        import torch

        load()  # once, before the threads
        self._local = threading.local()
        self._contexts = []
        self._lock = threading.Lock()
        self._device = torch.cuda.current_device()
        self._pool = ThreadPoolExecutor(max_workers=max(1, workers))

    def _context(self):
        import torch

        if not hasattr(self._local, "jp"):
            torch.cuda.set_device(self._device)
            self._local.stream = torch.cuda.Stream()
            self._local.jp = JpegPipeline(self._local.stream)
            with self._lock:
                self._contexts.append(self._local.jp)
        return self._local.jp, self._local.stream

    def filter_many(self, datas, radius: int, levels: int, flags: int = 0, quality: int = 90,
                    sampling: int = OP_JPEG_CSS_420) -> list:
        """JpegPipeline.filter over every JPEG byte string of `datas`;
        the encoded outputs in input order."""
        def one(data):
            jp, stream = self._context()
            return jp.filter(data, radius, levels, flags, quality, sampling, stream=stream)

        def some(chunk):
            jp, stream = self._context()
            return jp.filter_batch(chunk, radius, levels, flags, quality, sampling, stream=stream)

        if self._batch == 1:
            return list(self._pool.map(one, datas))
        datas = list(datas)
        chunks = [datas[i:i + self._batch] for i in range(0, len(datas), self._batch)]
        return [out for part in self._pool.map(some, chunks) for out in part]

    def close(self):
        self._pool.shutdown(wait=True)
        for jp in self._contexts:
            jp.close()
        self._contexts = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def filter_many(datas, radius: int, levels: int, flags: int = 0, quality: int = 90,
                sampling: int = OP_JPEG_CSS_420, workers: int = 4, batch: int = 8) -> list:
    """JpegPool(workers, batch).filter_many(...) for a one-off list of images."""
    with JpegPool(workers, batch) as pool:
        return pool.filter_many(datas, radius, levels, flags, quality, sampling)

def main(argv=None) -> int:
    """python -m paper_1405_1020_gb300.jpeg IN.jpg OUT.jpg [--radius R] [--levels L] ...

    Filters a JPEG file into another (section 3.2's ApplyOilPaintOnFile) and
    prints the decode, filter and encode times, as the paper's driver logs
    them."""
    import argparse
    import json

    p = argparse.ArgumentParser(description="oil-paint filter of a JPEG file, on the GPU")
    p.add_argument("input")
    p.add_argument("output")
    p.add_argument("--radius", type=int, default=5)
    p.add_argument("--levels", type=int, default=20)
    p.add_argument("--quality", type=int, default=90)
    p.add_argument("--sampling", choices=["444", "422", "420"], default="420")
    p.add_argument("--intdiv3", action="store_true", help="level from floor((R+G+B)/3)")
    p.add_argument("--literal", action="store_true", help="section 4's listing as printed")
    a = p.parse_args(argv)
    flags = (binding.OP_LEVEL_INTDIV3 if a.intdiv3 else 0) | (binding.OP_LITERAL if a.literal else 0)
    sampling = {"444": OP_JPEG_CSS_444, "422": OP_JPEG_CSS_422, "420": OP_JPEG_CSS_420}[a.sampling]
    with JpegPipeline() as jp:
        jp.filter_file(a.input, a.output, a.radius, a.levels, flags, a.quality, sampling)
        w, h, _ = jp.info(open(a.output, "rb").read())
        print(json.dumps({"width": w, "height": h, **jp.last_timing()}))
    return 0


if __name__ == "__main__":
    import sys

    sys.exit(main())
