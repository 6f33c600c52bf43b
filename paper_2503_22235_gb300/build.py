"""Build libwm.so (in tree, next to this file) from csrc/*.cu for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library with the CUDA runtime linked statically. No cmake, no torch
extension machinery: the library has a plain C ABI (include/wm.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libwm.so")
# The debug build: the same sources with WM_DEBUG_CHECKS=1, i.e. device-side
# checks of the attention windows, slab geometry and tail tiles that record
# WM_ERR_BOUNDS in the device status word and skip the access.
LIB_DEBUG = os.path.join(HERE, "libwm_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                     "-I" + os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libwm")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "wm.h"), __file__]


def _lib(debug: bool) -> str:
    return LIB_DEBUG if debug else LIB


def _flags(debug: bool):
    return NVCC_FLAGS + (["-DWM_DEBUG_CHECKS=1"] if debug else [])


def _source_hash(debug: bool = False) -> str:
    """sha256 over every input of the build (sources, headers, this script,
    the compiler flags) and the host architecture, so a library built from
    other sources, or on another machine, is never taken as current."""
    h = hashlib.sha256()
    h.update(platform.machine().encode())
    h.update(" ".join(_flags(debug)).encode())
    for p in sorted(_deps()):
        h.update(os.path.relpath(p, ROOT).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def up_to_date(debug: bool = False) -> bool:
    """True when the library exists and was linked from exactly the current sources."""
    lib, stamp = _lib(debug), _lib(debug) + ".sha256"
    if not os.path.exists(lib) or not os.path.exists(stamp):
        return False
    with open(stamp) as f:
        return f.read().strip() == _source_hash(debug)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link libwm.so (libwm_debug.so with debug=True); returns its
    path. Rebuilds unless the stamp beside the library records the hash of
    the current sources."""
    lib = _lib(debug)
    stamp = lib + ".sha256"
    if not force and up_to_date(debug):
        return lib
    digest = _source_hash(debug)
    nvcc = _nvcc()
    bdir = os.path.join(BUILD, "debug") if debug else BUILD
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    objs = [os.path.join(bdir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    flags = _flags(debug)

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r.returncode, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, zip(srcs, objs)))
    errors = [(s, out) for s, rc, out in results if rc != 0]
    if verbose:
        for s, rc, out in results:
            if out.strip():
                print(f"--- {os.path.basename(s)}\n{out}", file=sys.stderr)
    if errors:
        msg = "\n".join(f"--- {os.path.basename(s)}\n{out}" for s, out in errors)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    with open(stamp + ".tmp", "w") as f:
        f.write(digest + "\n")
    os.replace(stamp + ".tmp", stamp)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
