"""Python binding of the SeqCDC C ABI (``include/seqcdc.h``).

Argument marshalling only: each ``seqcdc_*`` function here forwards to the C
entry point of the same name in ``libseqcdc.so``, passing raw device pointers
taken from PyTorch tensors and the current CUDA stream.  PyTorch provides
device memory and streams; every step of the chunker runs in the library's
kernels.  There is no CPU fallback: if the library cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import threading
from dataclasses import dataclass

from . import _build

SEQCDC_OK = 0
SEQCDC_EINVAL = 1
SEQCDC_ECAPACITY = 2
SEQCDC_ECUDA = 3
SEQCDC_ETIMEOUT = 4
SEQCDC_ERANGE = 5

INCREASING = 0
DECREASING = 1


class SeqCDCError(RuntimeError):
    """A seqcdc entry point returned a non-zero status."""

    def __init__(self, status: int, where: str):
        super().__init__("%s: %s (status %d)" % (where, seqcdc_strerror(status), status))
        self.status = status


class Params(ctypes.Structure):
    """``seqcdc_params_t``: mode, seq_length, skip_trigger, skip_size, min, max."""

    _fields_ = [
        ("mode", ctypes.c_uint32),
        ("seq_length", ctypes.c_uint32),
        ("skip_trigger", ctypes.c_uint32),
        ("skip_size", ctypes.c_uint32),
        ("min_size", ctypes.c_uint64),
        ("max_size", ctypes.c_uint64),
    ]

    def astuple(self):
        return (self.mode, self.seq_length, self.skip_trigger, self.skip_size,
                self.min_size, self.max_size)

    def __repr__(self):
        return ("Params(mode=%d, seq_length=%d, skip_trigger=%d, skip_size=%d, "
                "min_size=%d, max_size=%d)" % self.astuple())


ALGO_AUTO = 0
ALGO_MAP = 1
ALGO_WALK = 2
WALK_MIN_FILES = 256   # SEQCDC_WALK_MIN_FILES: AUTO takes the chain walk from here
WALK_MIN_PIECES = 1024  # SEQCDC_WALK_MIN_PIECES: ... or from this many full pieces


class Tuning(ctypes.Structure):
    """``seqcdc_tuning_t``: segment_bytes, block_threads (segment map),
    algorithm (ALGO_AUTO / ALGO_MAP / ALGO_WALK), piece_bytes (chain walk);
    0 = default."""

    _fields_ = [("segment_bytes", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32),
                ("algorithm", ctypes.c_uint32),
                ("piece_bytes", ctypes.c_uint32)]


_lib = None
_lock = threading.Lock()

_SYMBOLS = ("seqcdc_params", "seqcdc_validate", "seqcdc_workspace_size",
            "seqcdc_chunk", "seqcdc_chunk_batch", "seqcdc_status",
            "seqcdc_strerror")


def load_library(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libseqcdc.so (building it first if needed) and declare its ABI."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB_PATH
        lib = ctypes.CDLL(path)
        P, T = ctypes.POINTER(Params), ctypes.POINTER(Tuning)
        u32, u64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
        lib.seqcdc_params.argtypes = [u32, u32, P]
        lib.seqcdc_params.restype = ctypes.c_int
        lib.seqcdc_validate.argtypes = [P]
        lib.seqcdc_validate.restype = ctypes.c_int
        lib.seqcdc_resolve_tuning.argtypes = [P, T, T]
        lib.seqcdc_resolve_tuning.restype = ctypes.c_int
        lib.seqcdc_workspace_size.argtypes = [P, u64, u64, T]
        lib.seqcdc_workspace_size.restype = ctypes.c_size_t
        lib.seqcdc_algorithm.argtypes = [P, u64, u64, ctypes.c_int, ctypes.c_size_t, T]
        lib.seqcdc_algorithm.restype = ctypes.c_int
        lib.seqcdc_chunk.argtypes = [P, vp, u64, vp, u64, vp, vp, ctypes.c_size_t, T, vp]
        lib.seqcdc_chunk.restype = ctypes.c_int
        lib.seqcdc_chunk_batch.argtypes = [P, vp, u64, vp, u64, vp, u64, vp, vp,
                                           ctypes.c_size_t, T, vp]
        lib.seqcdc_chunk_batch.restype = ctypes.c_int
        lib.seqcdc_chunk_noalloc.argtypes = [P, vp, u64, vp, u64, vp, vp, T, vp]
        lib.seqcdc_chunk_noalloc.restype = ctypes.c_int
        lib.seqcdc_status.argtypes = [vp, vp]
        lib.seqcdc_status.restype = ctypes.c_int
        lib.seqcdc_copy_ranges.argtypes = [vp, vp, vp, vp, vp, u64, vp]
        lib.seqcdc_copy_ranges.restype = ctypes.c_int
        lib.seqcdc_stats.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_uint32), u32]
        lib.seqcdc_stats.restype = ctypes.c_int
        lib.seqcdc_set_wait_limit_ns.argtypes = [u64]
        lib.seqcdc_set_wait_limit_ns.restype = u64
        lib.seqcdc_profile_events.argtypes = [vp, vp]
        lib.seqcdc_profile_events.restype = ctypes.c_int
        lib.seqcdc_fingerprint_batch.argtypes = [vp, u64, vp, u64, vp, vp, u64, vp, vp, vp]
        lib.seqcdc_fingerprint_batch.restype = ctypes.c_int
        lib.seqcdc_dedup_table_bytes.argtypes = [u64]
        lib.seqcdc_dedup_table_bytes.restype = ctypes.c_size_t
        lib.seqcdc_dedup.argtypes = [vp, vp, u64, vp, ctypes.c_size_t, vp, vp]
        lib.seqcdc_dedup.restype = ctypes.c_int
        lib.seqcdc_strerror.argtypes = [ctypes.c_int]
        lib.seqcdc_strerror.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != SEQCDC_OK:
        raise SeqCDCError(status, where)


def _tuning(tuning):
    if tuning is None:
        return None
    if isinstance(tuning, Tuning):
        return ctypes.byref(tuning)
    # (segment_bytes, block_threads[, algorithm[, piece_bytes]])
    return ctypes.byref(Tuning(*(int(v) for v in tuning)))


def _stream_handle(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return int(t.data_ptr()) if t is not None else 0


# ----------------------------------------------------------------------------
# Entry points (same names as the C ABI).
# ----------------------------------------------------------------------------
def seqcdc_params(expected_kib: int, mode: int = INCREASING) -> Params:
    """Paper parameter set for 4 / 8 / 16 KB expected chunks (Table I, Sec. VI)."""
    p = Params()
    _check(load_library().seqcdc_params(expected_kib, mode, ctypes.byref(p)),
           "seqcdc_params")
    return p


def make_params(mode, seq_length, skip_trigger, skip_size, min_size,
                max_size) -> Params:
    """A custom parameter set (validated by the library)."""
    p = Params(mode, seq_length, skip_trigger, skip_size, min_size, max_size)
    _check(load_library().seqcdc_validate(ctypes.byref(p)), "seqcdc_validate")
    return p


def seqcdc_validate(p: Params) -> int:
    return load_library().seqcdc_validate(ctypes.byref(p))


def seqcdc_resolve_tuning(p: Params, tuning=None) -> Tuning:
    """Segment size, block size and piece size a call with this tuning runs
    with (the algorithm as given)."""
    out = Tuning()
    _check(load_library().seqcdc_resolve_tuning(ctypes.byref(p), _tuning(tuning),
                                                ctypes.byref(out)),
           "seqcdc_resolve_tuning")
    return out


def seqcdc_workspace_size(p: Params, total_bytes: int, nfiles: int,
                          tuning=None) -> int:
    n = load_library().seqcdc_workspace_size(ctypes.byref(p), total_bytes,
                                             nfiles, _tuning(tuning))
    if n == 0:
        raise SeqCDCError(SEQCDC_EINVAL, "seqcdc_workspace_size")
    return n


def seqcdc_algorithm(p: Params, total_bytes: int, nfiles: int, batch: bool,
                     ws_bytes: int, tuning=None) -> int:
    """ALGO_MAP or ALGO_WALK: the path a call with these arguments takes."""
    a = load_library().seqcdc_algorithm(ctypes.byref(p), total_bytes, nfiles,
                                        1 if batch else 0, ws_bytes, _tuning(tuning))
    if a == 0:
        raise SeqCDCError(SEQCDC_EINVAL, "seqcdc_algorithm")
    return a


def seqcdc_chunk(p: Params, d_in, n: int, d_cuts, cap: int, d_count, d_ws,
                 ws_bytes: int, tuning=None, stream=None) -> None:
    """Raw entry point: tensors are device buffers the caller owns."""
    _check(load_library().seqcdc_chunk(
        ctypes.byref(p), _ptr(d_in), n, _ptr(d_cuts), cap, _ptr(d_count),
        _ptr(d_ws), ws_bytes, _tuning(tuning), _stream_handle(stream)),
        "seqcdc_chunk")


def seqcdc_chunk_batch(p: Params, d_data, total_bytes: int, d_offsets,
                       nfiles: int, d_cuts, cap: int, d_cut_offsets, d_ws,
                       ws_bytes: int, tuning=None, stream=None) -> None:
    """Raw entry point: tensors are device buffers the caller owns."""
    _check(load_library().seqcdc_chunk_batch(
        ctypes.byref(p), _ptr(d_data), total_bytes, _ptr(d_offsets), nfiles,
        _ptr(d_cuts), cap, _ptr(d_cut_offsets), _ptr(d_ws), ws_bytes,
        _tuning(tuning), _stream_handle(stream)), "seqcdc_chunk_batch")


SEQCDC_NOALLOC_SCRATCH_BYTES = 16 << 20


def seqcdc_chunk_noalloc(p: Params, d_in, n: int, d_cuts, cap: int, d_count,
                         d_status=None, tuning=None, stream=None) -> None:
    """Raw entry point that allocates nothing (fixed scratch inside the library).

    For callers that cannot allocate device memory; see include/seqcdc.h.
    """
    _check(load_library().seqcdc_chunk_noalloc(
        ctypes.byref(p), _ptr(d_in), n, _ptr(d_cuts), cap, _ptr(d_count),
        _ptr(d_status), _tuning(tuning), _stream_handle(stream)),
        "seqcdc_chunk_noalloc")


def seqcdc_copy_ranges(dst, src, dst_off, src_off, lens, stream=None) -> None:
    """Raw entry point: copy ranges ``src[src_off[i]:+lens[i]]`` to
    ``dst[dst_off[i]:]`` (tensors in device or pinned host memory; offsets
    and lengths as host arrays), each as one async copy on ``stream``."""
    import numpy as np
    a = np.ascontiguousarray(dst_off, dtype=np.uint64)
    b = np.ascontiguousarray(src_off, dtype=np.uint64)
    c = np.ascontiguousarray(lens, dtype=np.uint64)
    if not (a.size == b.size == c.size):
        raise ValueError("seqcdc_copy_ranges: offset and length arrays differ in size")
    _check(load_library().seqcdc_copy_ranges(
        _ptr(dst), _ptr(src), a.ctypes.data, b.ctypes.data, c.ctypes.data, int(a.size),
        _stream_handle(stream)), "seqcdc_copy_ranges")


def seqcdc_status(d_ws, stream=None) -> int:
    """Synchronise the stream; return the device-side status in the workspace."""
    return load_library().seqcdc_status(_ptr(d_ws), _stream_handle(stream))


STAT_NAMES = ("segments", "abnormal", "no_image", "lookback_waits", "inconsistent",
              "recomputed", "replayed", "lookback_steps")
WALK_STAT_NAMES = ("pieces", "piece_walk_chunks", "junction_walks", "junction_chunks",
                   "junctions_not_met", "inconsistent", "repaired", "windows")


def seqcdc_stats(d_ws, stream=None, walk: bool = False) -> dict:
    """Path counters of the last call that used workspace ``d_ws`` (named for
    the chain walk with ``walk=True``, else for the segment map)."""
    out = (ctypes.c_uint32 * 8)()
    _check(load_library().seqcdc_stats(_ptr(d_ws), _stream_handle(stream), out, 8),
           "seqcdc_stats")
    return dict(zip(WALK_STAT_NAMES if walk else STAT_NAMES, list(out)))


DEFAULT_WAIT_NS = 2_000_000_000   # SEQCDC_DEFAULT_WAIT_NS


def seqcdc_set_wait_limit_ns(ns: int) -> int:
    """Bound on device-side waits of later calls from this host thread;
    returns the previous bound (see include/seqcdc.h)."""
    return int(load_library().seqcdc_set_wait_limit_ns(int(ns)))


def seqcdc_profile_events(ev_begin=None, ev_end=None) -> None:
    """Bracket the segment kernel of later calls with two torch.cuda.Events."""
    h = (lambda e: int(e.cuda_event) if e is not None else None)
    _check(load_library().seqcdc_profile_events(h(ev_begin), h(ev_end)),
           "seqcdc_profile_events")


def seqcdc_strerror(status: int) -> str:
    try:
        return load_library().seqcdc_strerror(status).decode()
    except Exception:  # library not loadable: still describe the code
        return "status %d" % status


# ----------------------------------------------------------------------------
# Convenience wrappers that allocate outputs with PyTorch.
# ----------------------------------------------------------------------------
@dataclass
class BatchResult:
    cuts: "object"          # torch.uint64-compatible int64 tensor (device)
    cut_offsets: "object"   # int64 tensor (device), nfiles + 1


def _workspace(p, total, nfiles, tuning, device):
    import torch
    ws_bytes = seqcdc_workspace_size(p, total, nfiles, tuning)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=device)
    return ws, ws_bytes


def _on_stream(stream, device):
    """The stream a convenience call runs on (``stream`` or the current one),
    made current for the call: the tensors it allocates then belong to that
    stream in PyTorch's caching allocator, and the count it reads back is
    ordered after the kernels."""
    import torch
    return stream if stream is not None else torch.cuda.current_stream(device)


def _input_device(data, what: str):
    """The CUDA device that reads ``data``: its own for a CUDA tensor, the
    current one for a pinned host tensor (read in place by the kernels)."""
    import torch
    if data.dtype != torch.uint8:
        raise TypeError("%s needs uint8 data" % what)
    if data.is_cuda:
        return data.device
    if data.is_pinned():
        return torch.device("cuda", torch.cuda.current_device())
    raise TypeError("%s needs a CUDA tensor or a pinned host tensor" % what)


def chunk(data, p: Params, tuning=None, stream=None, check: bool = True):
    """Chunk one uint8 tensor; returns an int64 CUDA tensor of cut offsets.

    ``data`` is a CUDA tensor, or a pinned host tensor that the kernels read
    in place (only the windows the scan reaches cross to the GPU).
    """
    import torch
    dev = _input_device(data, "chunk()")
    data = data.contiguous().view(-1)
    n = data.numel()
    cap = n // p.min_size + 1
    st = _on_stream(stream, dev)
    with torch.cuda.stream(st):
        cuts = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
        count = torch.zeros(1, dtype=torch.int64, device=dev)
        ws, ws_bytes = _workspace(p, n, 1, tuning, dev)
        seqcdc_chunk(p, data, n, cuts, cap, count, ws, ws_bytes, tuning, st)
        if check:
            _check(seqcdc_status(ws, st), "seqcdc_chunk (device)")
        k = int(count.item())
    return cuts[:k]


def chunk_batch(data, offsets, p: Params, tuning=None, stream=None,
                check: bool = True) -> BatchResult:
    """Chunk a CSR batch: ``data`` uint8, ``offsets`` int64 (nfiles+1).

    ``data`` is a CUDA tensor, or a pinned host tensor that the kernels read
    in place; ``offsets`` a CUDA tensor, or a host tensor (copied to the
    device).  The results are CUDA tensors.
    """
    import torch
    dev = _input_device(data, "chunk_batch()")
    if offsets.dtype != torch.int64:
        raise TypeError("chunk_batch() needs int64 offsets")
    data = data.contiguous().view(-1)
    offsets = offsets.contiguous().view(-1)
    nfiles = offsets.numel() - 1
    total = data.numel()
    cap = total // p.min_size + nfiles
    st = _on_stream(stream, dev)
    with torch.cuda.stream(st):
        if not offsets.is_cuda:
            offsets = offsets.to(dev, non_blocking=offsets.is_pinned())
        cuts = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
        cut_offsets = torch.empty(nfiles + 1, dtype=torch.int64, device=dev)
        ws, ws_bytes = _workspace(p, total, nfiles, tuning, dev)
        seqcdc_chunk_batch(p, data, total, offsets, nfiles, cuts, cap, cut_offsets,
                           ws, ws_bytes, tuning, st)
        if check:
            _check(seqcdc_status(ws, st), "seqcdc_chunk_batch (device)")
        total_cuts = int(cut_offsets[-1].item())
    return BatchResult(cuts[:total_cuts], cut_offsets)


# ----------------------------------------------------------------------------
# Fingerprinting and deduplication (the step after chunking).
# ----------------------------------------------------------------------------
def seqcdc_fingerprint_batch(d_data, total_bytes: int, d_offsets, nfiles: int, d_cuts,
                             d_cut_offsets, ncuts: int, d_digests, d_sizes=None,
                             stream=None) -> None:
    """Raw entry point: SHA-256 of every chunk into ``d_digests`` (32 B each)."""
    _check(load_library().seqcdc_fingerprint_batch(
        _ptr(d_data), total_bytes, _ptr(d_offsets), nfiles, _ptr(d_cuts),
        _ptr(d_cut_offsets), ncuts, _ptr(d_digests), _ptr(d_sizes),
        _stream_handle(stream)), "seqcdc_fingerprint_batch")


def seqcdc_dedup_table_bytes(nchunks: int) -> int:
    return int(load_library().seqcdc_dedup_table_bytes(nchunks))


def seqcdc_dedup(d_digests, d_sizes, nchunks: int, d_table, table_bytes: int, d_out,
                 stream=None) -> None:
    """Raw entry point: distinct chunks / bytes into ``d_out`` (2 x uint64)."""
    _check(load_library().seqcdc_dedup(
        _ptr(d_digests), _ptr(d_sizes), nchunks, _ptr(d_table), table_bytes,
        _ptr(d_out), _stream_handle(stream)), "seqcdc_dedup")


def fingerprint(data, offsets, result: "BatchResult", stream=None):
    """SHA-256 of every chunk of a chunk_batch() result: (digests uint8 [n, 32],
    sizes int32 [n]) on the device."""
    import torch
    n = result.cuts.numel()
    dig = torch.empty((max(n, 1), 32), dtype=torch.uint8, device=data.device)
    sizes = torch.empty(max(n, 1), dtype=torch.int32, device=data.device)
    seqcdc_fingerprint_batch(data, data.numel(), offsets, offsets.numel() - 1,
                             result.cuts, result.cut_offsets, n, dig, sizes, stream)
    return dig[:n], sizes[:n]


def dedup(digests, sizes, stream=None):
    """(distinct chunks, distinct bytes) of fingerprinted chunks (synchronises)."""
    import torch
    n = digests.shape[0]
    tb = seqcdc_dedup_table_bytes(n)
    table = torch.empty(tb, dtype=torch.uint8, device=digests.device)
    out = torch.empty(2, dtype=torch.int64, device=digests.device)
    seqcdc_dedup(digests, sizes, n, table, tb, out, stream)
    c, b = out.cpu().tolist()
    return int(c), int(b)
