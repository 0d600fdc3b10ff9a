"""One stream chunked by several ranks (one GPU each).

The stream is cut into contiguous ranges, one per rank.  Each rank holds the
bytes of its range plus the max_size bytes after it, and:

1. walks its range's chain as if a chunk started at the range start (the
   spec walk), up to its exit, the first cut at or after the range end.  A
   chunk depends only on the bytes [c, c + max_size) after its start
   (Sec. IV), so the max_size bytes past the range end are enough;
2. sends its exit to the next rank, the one point-to-point exchange of the
   path (8 bytes), and receives the previous rank's exit.  That exit is
   where the true chain enters this range (rank 0's chain starts at byte 0);
3. walks from that entry (the junction walk) until it reaches a cut of its
   spec walk: from the meeting cut on, the two chains are the same.

If a junction reaches the range end without meeting (in long stretches
with no run ends, where every cut is forced), that rank's exit changes.  The
ranks then exchange again, until no exit changes.  Each round settles at
least one more rank, so there are at most `world` rounds; a MAX all-reduce of
a changed flag ends the loop.  A rank owns the cuts c with
start < c <= end (the last rank up to the stream end).

The chunking itself is ``chunk_fn(buf) -> int64 cut offsets`` relative to
``buf``'s first byte: the library's CUDA kernels in use
(``library_chunk_fn``), any exact chunker in tests.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Tuple

import numpy as np

from . import seqcdc

ChunkFn = Callable[[object], np.ndarray]


def split_ranges(n: int, world: int, align: int = 1 << 20) -> List[Tuple[int, int]]:
    """Contiguous ranges [start, end) of about n / world bytes each, with
    starts on multiples of ``align`` (the last range ends at n)."""
    world = max(1, int(world))
    bounds = [0]
    for r in range(1, world):
        b = (n * r // world) // align * align
        bounds.append(max(b, bounds[-1]))
    bounds.append(n)
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def held_bytes(start: int, end: int, n: int, p) -> Tuple[int, int]:
    """Bytes [lo, hi) of the stream a rank must hold for range [start, end)."""
    return start, min(end + int(p.max_size), n)


def spec_walk(buf, start: int, end: int, n: int, p, chunk_fn: ChunkFn) -> np.ndarray:
    """Cuts (absolute) of the chain that starts at ``start``, up to and
    including its exit, the first cut at or after ``end``.  ``buf`` holds the
    bytes [start, min(end + max_size, n)).

    The held bytes end at most max_size past ``end``; the chunk that covers
    ``end`` starts before it and so ends by its own max_size, inside them.
    Only a cut at the held end itself is the input end, which is right only
    when that end is the stream end, and then it is the last cut anyway."""
    hi = min(end + int(p.max_size), n)
    cuts = np.asarray(chunk_fn(buf[:hi - start]), dtype=np.int64) + start
    k = int(np.searchsorted(cuts, end, side="left"))
    return cuts[:k + 1]


def junction_walk(buf, start: int, end: int, n: int, x: int, spec: np.ndarray, p,
                  chunk_fn: ChunkFn, window: Optional[int] = None):
    """Walk the chain entering this range at cut ``x`` (absolute, start <= x)
    until it reaches a cut of ``spec`` or its exit (first cut >= end).

    Returns (cuts, met): ``cuts`` are the true cuts of the range from the
    entry on, with the exit last (the entry itself only if it lies inside
    the range, start < x); ``met`` says whether the walk met ``spec``.  The
    walk chunks windows of growing size from ``x``: a cut whose chunk start
    lies at least max_size before the window end does not depend on where
    the window ends."""
    mx = int(p.max_size)
    hi_held = min(end + mx, n)
    spec_set = set(spec.tolist())
    head = [x] if x > start else []
    if x >= end:   # entered at or past the range end: that cut is the exit
        return np.array(head if x > start else [x], dtype=np.int64), False
    if x == start:   # the spec walk started at the entry itself
        return spec.copy(), True
    if x in spec_set:
        k = int(np.searchsorted(spec, x))
        return np.concatenate([np.array(head, dtype=np.int64), spec[k + 1:]]), True
    w = window or 64 * mx
    while True:
        lo = x
        top = min(lo + w, hi_held)
        cuts = np.asarray(chunk_fn(buf[lo - start:top - start]), dtype=np.int64) + lo
        # cuts trusted: those whose chunk started at or before top - mx (or
        # all of them when the window reaches the held end)
        trusted = []
        prev = lo
        for c in cuts.tolist():
            if top < hi_held and prev > top - mx:
                break
            trusted.append(c)
            if c in spec_set:
                k = int(np.searchsorted(spec, c))
                return np.concatenate([np.array(head + trusted, dtype=np.int64),
                                       spec[k + 1:]]), True
            if c >= end:
                return np.array(head + trusted, dtype=np.int64), False
            prev = c
        if top >= hi_held:   # cannot happen: the chain leaves the range first
            raise RuntimeError("junction walk ran past the held bytes")
        w *= 2


def owned(cuts: np.ndarray, start: int, end: int) -> np.ndarray:
    """The cuts a range [start, end) owns: start < c <= end."""
    cuts = np.asarray(cuts, dtype=np.int64)
    return cuts[(cuts > start) & (cuts <= end)]


def chunk_stream_distributed(buf, start: int, end: int, n: int, p,
                             chunk_fn: Optional[ChunkFn] = None, device="cpu",
                             group=None) -> np.ndarray:
    """Run by every rank of the process group at once: this rank's range is
    [start, end) of a stream of n bytes (ranges contiguous, in rank order),
    ``buf`` holds its bytes [start, min(end + max_size, n)).  Returns the
    cuts (absolute) this rank owns; the ranks' results in rank order are the
    stream's cut list.  ``device`` holds the 8-byte exchange tensors (a CUDA
    device under NCCL)."""
    import torch
    import torch.distributed as dist
    fn = chunk_fn or library_chunk_fn(p)
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    spec = spec_walk(buf, start, end, n, p, fn)
    cuts = spec
    exit_ = int(spec[-1])
    entry_used = start if rank == 0 else -1
    for _ in range(world + 1):
        send = torch.tensor([exit_], dtype=torch.int64, device=device)
        recv = torch.zeros(1, dtype=torch.int64, device=device)
        req = dist.isend(send, rank + 1, group) if rank + 1 < world else None
        if rank > 0:
            dist.recv(recv, rank - 1, group)
        if req is not None:
            req.wait()
        changed = 0
        if rank > 0:
            x = int(recv.item())
            if x != entry_used:
                cuts, _ = junction_walk(buf, start, end, n, x, spec, p, fn)
                entry_used = x
                new_exit = int(cuts[-1])
                changed = int(new_exit != exit_)
                exit_ = new_exit
        flag = torch.tensor([changed], dtype=torch.int64, device=device)
        dist.all_reduce(flag, op=dist.ReduceOp.MAX, group=group)
        if int(flag.item()) == 0:
            return owned(cuts, start, end)
    raise RuntimeError("range exits did not settle")


def library_chunk_fn(p, tuning=None) -> ChunkFn:
    """``chunk_fn`` on the library's kernels: ``buf`` is a uint8 CUDA tensor
    (copied to an aligned buffer when a walk starts at an unaligned cut)."""
    def fn(buf):
        if buf.data_ptr() % 16:
            buf = buf.clone()
        return seqcdc.chunk(buf, p, tuning).cpu().numpy()
    return fn


def chunk_stream_ranges(bufs, ranges, n: int, p, chunk_fn: Optional[ChunkFn] = None):
    """The same rounds in one process over every range (``bufs[r]`` holds the
    bytes of range r as in ``chunk_stream_distributed``): the stream's cut
    list, and the number of exchange rounds it took."""
    fn = chunk_fn or library_chunk_fn(p)
    specs = [spec_walk(bufs[r], a, b, n, p, fn) for r, (a, b) in enumerate(ranges)]
    cuts = list(specs)
    exits = [int(s[-1]) for s in specs]
    used = [ranges[0][0]] + [-1] * (len(ranges) - 1)
    for rnd in range(len(ranges) + 1):
        sent = list(exits)   # what every rank sends this round
        changed = False
        for r in range(1, len(ranges)):
            x = sent[r - 1]
            if x != used[r]:
                a, b = ranges[r]
                cuts[r], _ = junction_walk(bufs[r], a, b, n, x, specs[r], p, fn)
                used[r] = x
                changed |= int(cuts[r][-1]) != exits[r]
                exits[r] = int(cuts[r][-1])
        if not changed:
            return np.concatenate([owned(c, a, b) for c, (a, b) in zip(cuts, ranges)]), rnd + 1
    raise RuntimeError("range exits did not settle")
