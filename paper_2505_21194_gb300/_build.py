"""Build the CUDA library ``libseqcdc.so`` in-tree with nvcc for sm_103a.

The library is the product path: every step of the chunker runs in its
kernels.  It is compiled next to its sources (``csrc/``) into ``_lib/`` and
loaded from there; nothing is installed into site-packages.
"""
from __future__ import annotations

import os
import shutil
import subprocess

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
SRC_DIR = os.path.join(PKG_DIR, "csrc")
INCLUDE_DIR = os.path.join(REPO_DIR, "include")
LIB_DIR = os.path.join(PKG_DIR, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libseqcdc.so")

SOURCES = ["seqcdc.cu", "walk.cu", "fingerprint.cu"]
HEADERS = ["common.cuh", "walk.h"]
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the SeqCDC CUDA library cannot be built")


def _inputs():
    files = [os.path.join(SRC_DIR, s) for s in SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE_DIR, "seqcdc.h"))
    return files


def is_stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libseqcdc.so if it is missing or older than its sources."""
    if not force and not is_stale():
        return LIB_PATH
    os.makedirs(LIB_DIR, exist_ok=True)
    nvcc = _nvcc()
    flags = [*ARCH_FLAGS, "-O3", "-lineinfo", "-std=c++17", "-I" + INCLUDE_DIR,
             "-Xcompiler", "-fPIC"]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    # Translation units compile in parallel, then one link.
    objs, procs = [], []
    for s in SOURCES:
        obj = os.path.join(LIB_DIR, s.replace(".cu", ".%d.o" % os.getpid()))
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc, *flags, "-c", "-o", obj,
                                       os.path.join(SRC_DIR, s)]))
    failed = [p.wait() for p in procs]
    try:
        if any(failed):
            raise subprocess.CalledProcessError(max(failed), "nvcc -c")
        tmp = LIB_PATH + ".%d.tmp" % os.getpid()
        subprocess.run([nvcc, *ARCH_FLAGS, "-shared", "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB_PATH)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB_PATH
