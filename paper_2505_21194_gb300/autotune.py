"""Launch tuning: which path, and its sizes, chosen by timing and cached.

Candidates are (segment bytes, threads, algorithm, piece bytes) tuples, the
fields of ``seqcdc_tuning_t``: the segment map with each segment size x block
size, and the chain walk with each piece size.  Each candidate is timed on
the caller's (device-resident) workload: the whole chunking call (all of its
kernels) with CUDA events on the launching stream, after warm-up, median of a
few runs.  The fastest (the library default when it is within 1 %, i.e.
within the timing noise) is stored in a JSON cache keyed by the GPU model and
SM count, the parameter set and the shape of the workload (single stream or
batch, the number of files and the median file size in powers of two), so a
later process on the same kind of GPU reuses it without timing.

Segments must be at least max_size bytes and the block's shared memory must
fit; pieces must be at least 4 x max_size (the library adjusts other values;
a candidate it would change is skipped).  Timing runs only the library's
CUDA kernels.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import threading
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

from . import seqcdc

SEGMENTS = (32768, 49152, 65536, 98304, 131072, 196608, 262144)
THREADS = (128, 256, 512)
PIECES = (262144, 524288, 786432, 1048576, 1572864, 2097152, 4194304)
CACHE_VERSION = "v2"
_lock = threading.Lock()


def default_cache_path() -> str:
    env = os.environ.get("SEQCDC_TUNING_CACHE")
    if env:
        return env
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "seqcdc_gb300", "tuning.json")


def workload_key(gpu_name: str, sm_count: int, p, sizes: Sequence[int]) -> str:
    """Cache key: GPU model and SM count, parameter set, workload shape."""
    sizes = np.asarray(sizes, dtype=np.int64)
    kind = "stream" if sizes.size <= 1 else "batch"
    med = int(np.median(sizes)) if sizes.size else 0
    bucket = int(math.log2(med)) if med > 0 else 0
    nbucket = int(math.log2(sizes.size)) if sizes.size > 0 else 0
    params = "%d-%d-%d-%d-%d-%d" % (p.mode, p.seq_length, p.skip_trigger, p.skip_size,
                                    p.min_size, p.max_size)
    return "%s|%s|sm%d|%s|%s|2^%d files|2^%d" % (CACHE_VERSION, gpu_name, sm_count, params,
                                                 kind, nbucket, bucket)


def candidates(p, segments: Iterable[int] = SEGMENTS, threads: Iterable[int] = THREADS,
               pieces: Iterable[int] = PIECES) -> List[Tuple[int, int, int, int]]:
    """Tuning tuples the library runs as given: segment-map (segment, threads)
    pairs, then chain-walk piece sizes."""
    out = []
    for L in segments:
        if L < p.max_size:
            continue
        for t in threads:
            eff = seqcdc.seqcdc_resolve_tuning(p, (L, t, seqcdc.ALGO_MAP, 0))
            if (eff.segment_bytes, eff.block_threads) == (L, t):
                out.append((L, t, seqcdc.ALGO_MAP, 0))
    for P in pieces:
        eff = seqcdc.seqcdc_resolve_tuning(p, (0, 0, seqcdc.ALGO_WALK, P))
        if eff.piece_bytes == P:
            out.append((0, 0, seqcdc.ALGO_WALK, P))
    return out


def default_candidate(p, nfiles: int, batch: bool = True,
                      total_bytes: int = 0) -> Tuple[int, int, int, int]:
    """The tuple a call with the library defaults runs as (AUTO resolved by
    the library's own rule, seqcdc_algorithm)."""
    eff = seqcdc.seqcdc_resolve_tuning(p)
    if seqcdc.seqcdc_algorithm(p, total_bytes, nfiles, batch, 1 << 62) == seqcdc.ALGO_WALK:
        return (0, 0, seqcdc.ALGO_WALK, eff.piece_bytes)
    return (eff.segment_bytes, eff.block_threads, seqcdc.ALGO_MAP, 0)


def load_cache(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(path: str, key: str, entry: dict) -> None:
    with _lock:
        d = load_cache(path)
        d[key] = entry
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        tmp = path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def pick_best(times: Dict[tuple, float], default: Optional[tuple] = None,
              tol: float = 0.01) -> tuple:
    """Fastest candidate.  Within ``tol`` of the fastest (timing noise), the
    library default wins if it is among them, else the smallest tuple (smaller
    segment, then fewer threads)."""
    best = min(times.values())
    near = [c for c in times if times[c] <= best * (1.0 + tol)]
    if default is not None and default in near:
        return default
    return min(near, key=lambda c: (tuple(c), times[c]))


def time_candidate(p, d_data, d_offsets, tuning: tuple, reps: int = 5,
                   warmup: int = 3, stream=None) -> float:
    """Median milliseconds of one chunking call (all kernels) on the sample."""
    import torch
    s = stream or torch.cuda.current_stream()
    total = d_data.numel()
    nfiles = d_offsets.numel() - 1
    cap = total // p.min_size + nfiles
    cuts = torch.empty(max(cap, 1), dtype=torch.int64, device=d_data.device)
    co = torch.empty(nfiles + 1, dtype=torch.int64, device=d_data.device)
    ws_bytes = seqcdc.seqcdc_workspace_size(p, total, nfiles, tuning)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=d_data.device)

    def once():
        seqcdc.seqcdc_chunk_batch(p, d_data, total, d_offsets, nfiles, cuts, cap, co,
                                  ws, ws_bytes, tuning, s)

    for _ in range(warmup):
        once()
    torch.cuda.synchronize(d_data.device)
    if seqcdc.seqcdc_status(ws, s) != seqcdc.SEQCDC_OK:
        raise seqcdc.SeqCDCError(seqcdc.seqcdc_status(ws, s), "autotune")
    ms = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        once()
        b.record(s)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def autotune(p, d_data, d_offsets, cache_path: Optional[str] = None,
             cands: Optional[List[tuple]] = None,
             timer: Optional[Callable] = None, force: bool = False) -> tuple:
    """Best tuning tuple (segment bytes, threads, algorithm, piece bytes) for
    this kind of workload on this GPU.

    ``d_data`` (uint8) and ``d_offsets`` (int64, CSR) are the device-resident
    workload (or a sample of it); a single stream is ``offsets = [0, n]``.
    The result is cached at ``cache_path`` (default: ``default_cache_path()``).
    """
    import torch
    path = cache_path or default_cache_path()
    props = torch.cuda.get_device_properties(d_data.device)
    sizes = np.diff(d_offsets.cpu().numpy())
    key = workload_key(props.name, props.multi_processor_count, p, sizes)
    if not force:
        hit = load_cache(path).get(key)
        if hit and "tuning" in hit:
            return tuple(int(v) for v in hit["tuning"])
    cands = cands or candidates(p)
    timer = timer or time_candidate
    times = {tuple(c): timer(p, d_data, d_offsets, tuple(c)) for c in cands}
    best = pick_best(times, default_candidate(p, int(sizes.size), True, int(sizes.sum())))
    store_cache(path, key, {"tuning": list(best), "ms": times[best],
                            "sample_bytes": int(d_data.numel()),
                            "timed": {"x".join(str(v) for v in c): round(t, 4)
                                      for c, t in times.items()}})
    return best
