"""Builds the CUDA library paper_1405_1020_gb300/liboilpaint.so for sm_103a.

Six translation units (the kernels, the straight-line difference-histogram
kernels with two, four and eight columns per thread, the C ABI, and the
allocation-free entry point with its device scratch array) are compiled in
parallel with nvcc and linked into one shared library with the CUDA runtime linked statically, so
the library needs nothing but the NVIDIA driver at run time.  The library is
built in-tree (the package directory) and git-ignored.

build_jpeg() then builds liboilpaint_jpeg.so, the decode -> filter -> encode
pipeline (include/oilpaint_jpeg.h): one host translation unit linked against
liboilpaint.so (found beside it at run time) and the toolkit's nvJPEG.  It is
skipped, with a note, when the toolkit has no nvJPEG; the filter library does
not depend on it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

CSRC = os.path.dirname(os.path.abspath(__file__))
PKG = os.path.dirname(CSRC)
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "liboilpaint.so")
SOURCES = [
    "oilpaint_kernels.cu", "oilpaint_delta2.cu", "oilpaint_delta4.cu", "oilpaint_delta8.cu",
    "oilpaint_api.cu",
    "oilpaint_noalloc.cu",
]
HEADERS = ["oilpaint_device.cuh", "oilpaint_internal.h", "oilpaint_deltak.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liboilpaint.so")


CHECKED_LIB = os.path.join(PKG, "liboilpaint_checked.so")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps += [os.path.join(INCLUDE, "oilpaint.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), checked: bool = False) -> str:
    """Compile and link the library if missing or older than its sources.
    checked=True builds the bounds-checking variant liboilpaint_checked.so
    (OPK_CHECKED: every shared-memory, pixel and TMA access is range-checked,
    violations are reported as OP_E_BOUNDS instead of faulting)."""
    lib = CHECKED_LIB if checked else LIB
    if not force and not _stale(lib):
        return lib
    if checked:
        extra_flags = tuple(extra_flags) + ("-DOPK_CHECKED=1",)
    nvcc = _nvcc()
    bdir = os.path.join(PKG, "_build_checked" if checked else "_build")
    os.makedirs(bdir, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                            text=True)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if verbose and out:
            print(out)
        if p.returncode != 0:
            failed.append((src, out))
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xlinker", "-soname=" + os.path.basename(lib), "-o", tmp,
           *objs]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


JPEG_LIB = os.path.join(PKG, "liboilpaint_jpeg.so")
JPEG_SOURCE = "oilpaint_jpeg.cu"


def nvjpeg_dirs():
    """(include dir, library dir) of the toolkit's nvJPEG, or None."""
    home = os.path.dirname(os.path.dirname(os.path.realpath(_nvcc())))
    inc = os.path.join(home, "include")
    if not os.path.exists(os.path.join(inc, "nvjpeg.h")):
        return None
    cands = [os.path.join(home, "lib64"), os.path.join(home, "lib")]
    tdir = os.path.join(home, "targets")
    if os.path.isdir(tdir):
        cands += [os.path.join(tdir, t, "lib") for t in sorted(os.listdir(tdir))]
    for d in cands:
        if os.path.exists(os.path.join(d, "libnvjpeg.so")):
            return inc, d
    return None


def build_jpeg(force: bool = False, verbose: bool = False):
    """Build liboilpaint_jpeg.so if missing or stale; None when nvJPEG is absent."""
    dirs = nvjpeg_dirs()
    if dirs is None:
        print("oilpaint: nvJPEG not found in the CUDA toolkit; liboilpaint_jpeg.so not built")
        return None
    inc, libdir = dirs
    deps = [os.path.join(CSRC, JPEG_SOURCE), os.path.join(INCLUDE, "oilpaint_jpeg.h"),
            os.path.join(INCLUDE, "oilpaint.h"), os.path.abspath(__file__), LIB]
    if (not force and os.path.exists(JPEG_LIB)
            and all(os.path.getmtime(d) <= os.path.getmtime(JPEG_LIB) for d in deps)):
        return JPEG_LIB
    nvcc = _nvcc()
    bdir = os.path.join(PKG, "_build")
    os.makedirs(bdir, exist_ok=True)
    obj = os.path.join(bdir, JPEG_SOURCE.replace(".cu", ".o"))
    cmd = [nvcc, *ARCH, *FLAGS, "-I", inc, "-c", os.path.join(CSRC, JPEG_SOURCE), "-o", obj]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    tmp = JPEG_LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xlinker", "-soname=liboilpaint_jpeg.so", "-o", tmp, obj,
           "-L", PKG, "-loilpaint", "-L", libdir, "-lnvjpeg",
           "-Xlinker", "-rpath=$ORIGIN", "-Xlinker", "-rpath=" + libdir]
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, JPEG_LIB)
    return JPEG_LIB


ALU_PROBE = os.path.join(PKG, "alu_probe")
SMEM_UPDATE_PROBE = os.path.join(PKG, "smem_update_probe")


def _build_probe(name: str, exe: str, force: bool) -> str:
    src = os.path.join(CSRC, name + ".cu")
    if (not force and os.path.exists(exe)
            and os.path.getmtime(exe) >= os.path.getmtime(src)):
        return exe
    tmp = exe + f".tmp{os.getpid()}"
    subprocess.run([_nvcc(), *ARCH, "-O3", "-std=c++17", src, "-o", tmp], check=True)
    os.replace(tmp, exe)
    return exe


def build_alu_probe(force: bool = False) -> str:
    """Build the integer-ALU throughput probe (alu_probe.cu), a standalone
    program that measures the roofline denominator of the filter kernels."""
    return _build_probe("alu_probe", ALU_PROBE, force)


def build_smem_update_probe(force: bool = False) -> str:
    """Build the shared-memory bin-update probe (smem_update_probe.cu), a
    standalone program that times a histogram bin update as load-add-store
    and as shared-memory reductions."""
    return _build_probe("smem_update_probe", SMEM_UPDATE_PROBE, force)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
    if "--checked" not in sys.argv:
        print(build_jpeg(force="--force" in sys.argv, verbose="-v" in sys.argv))
