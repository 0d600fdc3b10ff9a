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

SOURCES = ["seqcdc.cu"]
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the SeqCDC CUDA library cannot be built")


def _inputs():
    files = [os.path.join(SRC_DIR, s) for s in SOURCES]
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
    tmp = LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = [_nvcc(), *ARCH_FLAGS, "-O3", "-lineinfo", "-std=c++17",
           "-I" + INCLUDE_DIR, "-shared", "-Xcompiler", "-fPIC",
           "-o", tmp] + [os.path.join(SRC_DIR, s) for s in SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH
