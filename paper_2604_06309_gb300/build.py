"""Build libdmfe.so in-tree for sm_103a (nvcc, one -gencode, translation units in parallel)."""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libdmfe.so")
CHECKED_LIB = os.path.join(PKG, "libdmfe_checked.so")

SOURCES = ["kernels_hi.cu", "kernels_df.cu", "kernels_step.cu", "api.cu", "host_grid.cpp", "noalloc.cu", "batch.cu", "server.cu", "graph.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I" + os.path.join(ROOT, "include")]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            return cand
        raise RuntimeError("nvcc not found: libdmfe.so cannot be built")
    return exe


def _compile(src, extra, tag=""):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + tag + ".o")
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj, r.stderr


def build(verbose=False, extra=(), checked=False):
    """Compile every translation unit and link libdmfe.so next to this file; checked=True
    builds libdmfe_checked.so instead, with the bounds checks of -DDMFE_CHECKED."""
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra) + (["-DDMFE_CHECKED"] if checked else [])
    tag = "_checked" if checked else ""
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, tag), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, err in results:
            if err.strip():
                sys.stderr.write(err)
    lib = CHECKED_LIB if checked else LIB
    tmp = lib + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [],
                checked="--checked" in sys.argv))
