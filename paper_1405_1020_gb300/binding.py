"""ctypes binding of include/oilpaint.h -- argument marshalling only.

Every function has the name and the argument order of the C entry point and
returns what it returns (status codes are plain ints; handles are opaque
ints).  Device pointers are ints (e.g. ``tensor.data_ptr()``), streams are
ints (``torch.cuda.current_stream().cuda_stream``) or None.

The library is ``liboilpaint.so`` next to this file, built by
``__graft_entry__.build()`` (or ``python paper_1405_1020_gb300/csrc/build.py``).
There is no fallback: if it is missing, every call raises ``OilPaintError``.
"""
from __future__ import annotations

import ctypes
import os

OP_OK = 0
OP_E_INVALID = -1
OP_E_CUDA = -2
OP_E_NOMEM = -3
OP_E_TIMEOUT = -4
OP_E_UNSUPPORTED = -5
OP_E_BOUNDS = -6  # the bounds-checking build found and skipped an out-of-range access

OP_LEVEL_PAPER = 0
OP_LEVEL_INTDIV3 = 1
OP_LITERAL = 2  # flag bit: the section-4 listing as printed
OP_LITERAL_MAX_LEVELS = 254
OP_FUSED_PACK = 4  # flag bit: pack in the filter's shared memory, no prepass launch

OP_MAX_RADIUS = 44
OP_MAX_LEVELS = 256
OP_MAX_DIM = 65535
OP_NOALLOC_MAX_WORDS = 4 * 1024 * 1024

_PKG = os.path.dirname(os.path.abspath(__file__))
# OPK_LIBRARY=checked loads the bounds-checking build (liboilpaint_checked.so)
LIB_PATH = os.path.join(_PKG, "liboilpaint_checked.so" if os.environ.get("OPK_LIBRARY") == "checked"
                        else "liboilpaint.so")

# every symbol include/oilpaint.h declares
EXPORTS = (
    "op_create", "op_create_ex", "op_last_error", "op_status_string", "op_get_config",
    "op_set_config", "op_default_config", "op_tune_table_set",
    "op_batch_tune_table_set", "op_workspace_size",
    "op_set_workspace", "op_run", "op_run_host", "op_run_host_async", "op_set_profile_event",
    "op_sync_status",
    "op_destroy",
    "op_batch_create", "op_batch_get_config", "op_batch_group_count", "op_batch_get_group",
    "op_batch_workspace_size",
    "op_batch_set_workspace", "op_batch_set",
    "op_batch_run", "op_batch_capture", "op_batch_launch_graph", "op_batch_sync_status",
    "op_batch_destroy", "op_selftest_wait_timeout", "op_run_noalloc",
)


class OilPaintError(RuntimeError):
    """A failed call (status in .status) or a missing library."""

    def __init__(self, msg: str, status: int | None = None):
        super().__init__(msg)
        self.status = status


class op_config_t(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_uint32), ("tile_h", ctypes.c_uint32),
                ("chunk_rows", ctypes.c_uint32), ("prefetch", ctypes.c_uint32),
                ("cols_per_thread", ctypes.c_uint32), ("path", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {f: int(getattr(self, f)) for f, _ in self._fields_}

    @classmethod
    def make(cls, tile_w: int, tile_h: int = 0, chunk_rows: int = 8, prefetch: int = 2,
             cols_per_thread: int = 1, path: int = 0):
        return cls(tile_w, tile_h, chunk_rows, prefetch, cols_per_thread, path)


class op_image_t(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("stride", ctypes.c_uint32), ("bpp", ctypes.c_uint32),
                ("radius", ctypes.c_int32), ("levels", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("out_stride", ctypes.c_uint32)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liboilpaint.so (once) and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OilPaintError(f"{path} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    u32, i32, u64 = ctypes.c_uint32, ctypes.c_int32, ctypes.c_uint64
    vp, sz, ci = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
    cfgp = ctypes.POINTER(op_config_t)
    sig = {
        "op_create": (vp, [u32, u32, u32, i32, u32]),
        "op_create_ex": (vp, [u32, u32, u32, u32, i32, u32, u32]),
        "op_last_error": (ci, []),
        "op_status_string": (ctypes.c_char_p, [ci]),
        "op_get_config": (ci, [vp, cfgp]),
        "op_set_config": (ci, [vp, cfgp]),
        "op_default_config": (ci, [i32, u32, cfgp]),
        "op_tune_table_set": (ci, [i32, u32, cfgp]),
        "op_batch_tune_table_set": (ci, [i32, u32, cfgp]),
        "op_workspace_size": (sz, [vp]),
        "op_set_workspace": (ci, [vp, vp, sz]),
        "op_run": (ci, [vp, vp, vp, vp]),
        "op_run_host": (ci, [vp, vp, vp, vp]),
        "op_run_host_async": (ci, [vp, vp, vp, vp]),
        "op_set_profile_event": (ci, [vp, vp]),
        "op_sync_status": (ci, [vp, vp]),
        "op_destroy": (ci, [vp]),
        "op_batch_create": (vp, [u32, u64, i32, u32, cfgp]),
        "op_batch_get_config": (ci, [vp, cfgp]),
        "op_batch_group_count": (ci, [vp]),
        "op_batch_get_group": (ci, [vp, u32, cfgp, ctypes.POINTER(i32), ctypes.POINTER(u32)]),
        "op_batch_workspace_size": (sz, [vp]),
        "op_batch_set_workspace": (ci, [vp, vp, sz]),
        "op_batch_set": (ci, [vp, ctypes.POINTER(op_image_t), u32, vp]),
        "op_batch_run": (ci, [vp, vp]),
        "op_batch_capture": (ci, [vp, vp]),
        "op_batch_launch_graph": (ci, [vp, vp]),
        "op_batch_sync_status": (ci, [vp, vp]),
        "op_batch_destroy": (ci, [vp]),
        "op_selftest_wait_timeout": (ci, [u64, vp]),
        "op_run_noalloc": (ci, [vp, vp, u32, u32, u32, u32, i32, u32, u32, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().op_status_string(status).decode()


def check(status: int, what: str = "call") -> int:
    """Raise OilPaintError unless status == OP_OK."""
    if status != OP_OK:
        raise OilPaintError(f"{what} failed: {status_string(status)} ({status})", status)
    return status


# ---- same-named wrappers (argument marshalling only) ----------------------

def op_create(width, height, stride, radius, levels):
    return load().op_create(width, height, stride, radius, levels)


def op_create_ex(width, height, stride, bpp, radius, levels, flags=OP_LEVEL_PAPER):
    return load().op_create_ex(width, height, stride, bpp, radius, levels, flags)


def op_last_error():
    return load().op_last_error()


def op_status_string(status):
    return status_string(status)


def op_get_config(op, cfg: op_config_t):
    return load().op_get_config(op, ctypes.byref(cfg))


def op_set_config(op, cfg: op_config_t):
    return load().op_set_config(op, ctypes.byref(cfg))


def op_default_config(radius, levels, cfg: op_config_t):
    return load().op_default_config(radius, levels, ctypes.byref(cfg))


def op_tune_table_set(radius, levels, cfg: op_config_t):
    return load().op_tune_table_set(radius, levels, ctypes.byref(cfg))


def op_batch_tune_table_set(max_radius, max_levels, cfg: op_config_t | None):
    """cfg None removes the entry."""
    return load().op_batch_tune_table_set(max_radius, max_levels,
                                          None if cfg is None else ctypes.byref(cfg))


def op_workspace_size(op):
    return load().op_workspace_size(op)


def op_set_workspace(op, d_ws, nbytes):
    return load().op_set_workspace(op, d_ws, nbytes)


def op_run(op, d_in, d_out, stream=None):
    return load().op_run(op, d_in, d_out, stream)


def op_run_host(op, h_in, h_out, stream=None):
    return load().op_run_host(op, h_in, h_out, stream)


def op_run_host_async(op, h_in, h_out, stream=None):
    return load().op_run_host_async(op, h_in, h_out, stream)


def op_set_profile_event(op, event):
    return load().op_set_profile_event(op, event)


def op_sync_status(op, stream=None):
    return load().op_sync_status(op, stream)


def op_destroy(op):
    return load().op_destroy(op)


def op_batch_create(max_images, max_pixels, max_radius, max_levels, cfg: op_config_t | None = None):
    return load().op_batch_create(max_images, max_pixels, max_radius, max_levels,
                                  ctypes.byref(cfg) if cfg is not None else None)


def op_batch_get_config(b, cfg: op_config_t):
    return load().op_batch_get_config(b, ctypes.byref(cfg))


def op_batch_group_count(b):
    return load().op_batch_group_count(b)


def op_batch_get_group(b, group: int, cfg: op_config_t, max_radius, max_levels):
    """max_radius / max_levels: ctypes.c_int32 / c_uint32 (or None)."""
    return load().op_batch_get_group(b, group, ctypes.byref(cfg),
                                     None if max_radius is None else ctypes.byref(max_radius),
                                     None if max_levels is None else ctypes.byref(max_levels))


def op_batch_workspace_size(b):
    return load().op_batch_workspace_size(b)


def op_batch_set_workspace(b, d_ws, nbytes):
    return load().op_batch_set_workspace(b, d_ws, nbytes)


def op_batch_set(b, images, n, stream=None):
    return load().op_batch_set(b, images, n, stream)


def op_batch_run(b, stream=None):
    return load().op_batch_run(b, stream)


def op_batch_capture(b, stream=None):
    return load().op_batch_capture(b, stream)


def op_batch_launch_graph(b, stream=None):
    return load().op_batch_launch_graph(b, stream)


def op_batch_sync_status(b, stream=None):
    return load().op_batch_sync_status(b, stream)


def op_batch_destroy(b):
    return load().op_batch_destroy(b)


def op_selftest_wait_timeout(timeout_ns, stream=None):
    return load().op_selftest_wait_timeout(timeout_ns, stream)


def op_run_noalloc(d_in, d_out, width, height, stride, bpp, radius, levels,
                   flags=OP_LEVEL_PAPER, stream=None):
    return load().op_run_noalloc(d_in, d_out, width, height, stride, bpp, radius, levels, flags,
                                 stream)
