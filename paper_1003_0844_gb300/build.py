"""Build the CUDA library in-tree: libfstat.so next to this file.

Each translation unit is compiled for sm_103a in parallel, then linked into a
shared library with the C ABI of include/fstat.h.  Run as a module or call
build().
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfstat.so")
SOURCES = ["fs_api.cu", "fs_fft64.cu", "fs_prep.cu", "fs_search32.cu", "fs_search64.cu", "fs_passes_small.cu",
           "fs_passes_mid.cu", "fs_passes_large.cu", "fs_passes_batch.cu", "fs_passes_ib.cu", "fs_passes_lat.cu",
           "fs_passes_lat_wide.cu", "fs_batch.cu", "fs_refine.cu", "fs_adjoint.cu", "fs_host.cu", "fs_grid.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
                   "-Xcompiler", "-fvisibility=hidden"] + list(extra)


def _compile(src: str, verbose: bool, extra, out_dir=OUT_DIR, src_dir=CSRC) -> str:
    obj = os.path.join(out_dir, os.path.splitext(src)[0] + ".o")
    srcp = os.path.join(src_dir, src)
    deps = [srcp] + [os.path.join(src_dir, h) for h in os.listdir(src_dir) if h.endswith((".h", ".cuh"))]
    deps.append(os.path.join(HERE, "..", "include", "fstat.h"))
    if os.path.exists(obj) and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
        return obj
    cmd = [nvcc()] + _flags(extra) + ["-c", srcp, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def build(verbose: bool = False, extra=(), lib: str = LIB, out_dir: str = OUT_DIR, src_dir: str = CSRC) -> str:
    """Compile and link; `extra` nvcc flags, `lib`/`out_dir` select another output,
    `src_dir` another copy of the sources (it must sit two levels below include/)."""
    os.makedirs(out_dir, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, extra, out_dir, src_dir), SOURCES))
    LIB_ = lib
    if os.path.exists(LIB_) and all(os.path.getmtime(LIB_) >= os.path.getmtime(o) for o in objs):
        return LIB_
    tmp = LIB_ + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB_)
    return LIB_


DEBUG_DIR = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_DIR, "libfstat_debug.so")


def build_debug(verbose: bool = False) -> str:
    """The debug build (-DFS_DEBUG) beside the release library: the transform
    kernels check every workspace and output index against its buffer (an index
    outside latches FS_ERR_CORRUPT and skips the access) and the search
    workspaces carry guard words around the transform ring and the queue
    counters, checked after every search.  Load it with FSTAT_LIB or
    fstat.load_library(path)."""
    return build(verbose=verbose, extra=["-DFS_DEBUG"], lib=DEBUG_LIB, out_dir=DEBUG_DIR)


if __name__ == "__main__":
    print(build_debug(verbose="-v" in sys.argv) if "--debug" in sys.argv else build(verbose="-v" in sys.argv))
