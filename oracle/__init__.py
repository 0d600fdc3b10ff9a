"""Plain CPU SeqCDC oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library (``paper_2505_21194_gb300``)
never imports it, and this package imports nothing from the library: the two
share no code, header, table or constant.

Two independent formulations of the same chunker live here:

* ``seqcdc_oracle.c`` -- the state machine of Sec. III (boundary runs of
  Sec. III.A, sub-minimum region of Sec. III.B, content-defined skipping of
  Sec. III.C, maximum chunk size of Sec. IV) as a byte-at-a-time C loop,
  wrapped here with ctypes (``chunk``, ``chunk_batch``).
* ``declarative.py`` -- the same rules restated from prefix counts (run
  lengths and cumulative opposing-pair counts) and searches, in plain Python,
  used to pin the C loop by brute force on tiny inputs.

The parameter presets in ``presets()`` restate Table I of the paper and the
minimum/maximum rule of Sec. VI (1/2x and 2x the expected size; 1 KB minimum
for the 4 KB setting), with KB read as 1024 bytes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seqcdc_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")

INCREASING = 0
DECREASING = 1


@dataclass(frozen=True)
class Params:
    """SeqCDC parameters (Sec. III, Table I).  ``skip_trigger == 0`` = no skip."""

    mode: int
    seq_length: int
    skip_trigger: int
    skip_size: int
    min_size: int
    max_size: int


def presets(expected_kib: int, mode: int = INCREASING) -> Params:
    """Table I (SeqLength, SkipTrigger, SkipSize) and Sec. VI min/max sizes."""
    table = {4: (5, 55, 256), 8: (5, 50, 256), 16: (5, 50, 512)}
    if expected_kib not in table:
        raise ValueError("the paper gives parameters for 4, 8 and 16 KB only")
    seq, trig, skip = table[expected_kib]
    avg = expected_kib * 1024
    mn = 1024 if expected_kib == 4 else avg // 2
    return Params(mode, seq, trig, skip, mn, 2 * avg)


class _CParams(ctypes.Structure):
    _fields_ = [
        ("mode", ctypes.c_uint32),
        ("seq_length", ctypes.c_uint32),
        ("skip_trigger", ctypes.c_uint32),
        ("skip_size", ctypes.c_uint32),
        ("min_size", ctypes.c_uint64),
        ("max_size", ctypes.c_uint64),
    ]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into ``oracle/_build``; return its path."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall",
                    "-Werror", "-o", tmp, _SRC], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_chunk.restype = ctypes.c_int64
            lib.oracle_chunk.argtypes = [
                ctypes.POINTER(_CParams), ctypes.c_void_p, ctypes.c_uint64,
                ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
            lib.oracle_chunk_batch.restype = ctypes.c_int64
            lib.oracle_chunk_batch.argtypes = [
                ctypes.POINTER(_CParams), ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64,
                ctypes.c_void_p]
            _lib = lib
    return _lib


def _cparams(p: Params) -> _CParams:
    return _CParams(p.mode, p.seq_length, p.skip_trigger, p.skip_size,
                    p.min_size, p.max_size)


def _as_u8(data) -> np.ndarray:
    a = np.ascontiguousarray(np.frombuffer(data, dtype=np.uint8)
                             if isinstance(data, (bytes, bytearray, memoryview))
                             else data)
    if a.dtype != np.uint8:
        raise TypeError("oracle input must be uint8 bytes")
    return a.reshape(-1)


def chunk(data, p: Params, return_examined: bool = False):
    """Chunk end offsets (uint64, strictly increasing, last == len) of ``data``."""
    b = _as_u8(data)
    n = b.size
    cap = n // max(p.min_size, 1) + 1
    cuts = np.empty(cap, dtype=np.uint64)
    examined = ctypes.c_uint64(0)
    k = _load().oracle_chunk(ctypes.byref(_cparams(p)), b.ctypes.data, n,
                             cuts.ctypes.data, cap, ctypes.addressof(examined))
    if k < 0:
        raise ValueError("oracle rejected the input (status %d)" % k)
    out = cuts[:k].copy()
    return (out, int(examined.value)) if return_examined else out


def chunk_batch(data, offsets: Sequence[int], p: Params):
    """Chunk every file of a CSR batch; returns (cuts, cut_offsets).

    File f is ``data[offsets[f]:offsets[f+1]]``; its cuts are relative to the
    file start and sit in ``cuts[cut_offsets[f]:cut_offsets[f+1]]``.
    """
    b = _as_u8(data)
    offs = np.ascontiguousarray(offsets, dtype=np.uint64)
    nfiles = offs.size - 1
    sizes = np.diff(offs.astype(np.int64))
    cap = int((sizes // max(p.min_size, 1) + 1).sum()) if nfiles > 0 else 0
    cuts = np.empty(max(cap, 1), dtype=np.uint64)
    cut_offsets = np.empty(nfiles + 1, dtype=np.uint64)
    k = _load().oracle_chunk_batch(ctypes.byref(_cparams(p)), b.ctypes.data,
                                   offs.ctypes.data, nfiles, cuts.ctypes.data,
                                   cap, cut_offsets.ctypes.data)
    if k < 0:
        raise ValueError("oracle rejected the batch (status %d)" % k)
    return cuts[:k].copy(), cut_offsets


def chunk_batch_threaded(data, offsets: Sequence[int], p: Params,
                         threads: int):
    """``chunk_batch`` with whole files handed out to ``threads`` host threads.

    Each file is still chunked by the single-threaded loop; ctypes releases
    the GIL during the C call, so files run concurrently.  Returns the same
    (cuts, cut_offsets) as ``chunk_batch``.
    """
    from concurrent.futures import ThreadPoolExecutor

    b = _as_u8(data)
    offs = np.asarray(offsets, dtype=np.int64)
    nfiles = offs.size - 1
    results = [None] * nfiles

    def work(f):
        results[f] = chunk(b[offs[f]:offs[f + 1]], p)

    with ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        list(ex.map(work, range(nfiles)))
    counts = np.array([r.size for r in results], dtype=np.uint64)
    cut_offsets = np.zeros(nfiles + 1, dtype=np.uint64)
    np.cumsum(counts, out=cut_offsets[1:])
    cuts = (np.concatenate(results) if nfiles else np.empty(0, np.uint64))
    return cuts.astype(np.uint64), cut_offsets


def chunk_stream(blocks, p: Params):
    """Chunk a stream delivered as an iterable of uint8 blocks.

    Uses the prefix property of the chunker: every cut of ``x[:m]`` except the
    final one (== m) is also a cut of any longer ``x``.  Bytes after the last
    proven cut are carried into the next block.  Yields absolute cut offsets
    as uint64 arrays.
    """
    carry = np.empty(0, dtype=np.uint8)
    base = 0
    for blk in blocks:
        buf = np.concatenate([carry, _as_u8(blk)]) if carry.size else _as_u8(blk)
        cuts = chunk(buf, p)
        if cuts.size > 1:
            keep = cuts[:-1]
            yield keep + np.uint64(base)
            last = int(keep[-1])
            carry = buf[last:].copy()
            base += last
        else:
            carry = buf.copy()
    if carry.size:
        yield chunk(carry, p) + np.uint64(base)
