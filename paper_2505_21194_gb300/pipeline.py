"""Chunking of host-resident data with the copies overlapped.

``chunk_batch_host`` takes a CSR batch in pinned host memory, splits it into
pieces of whole files, and pipelines each piece through a copy stream (host to
device), a compute stream (``seqcdc_chunk_batch``) and back (cut lists to
pinned host memory), with a few device slots in rotation: while piece k is
chunked, piece k+1 is copied in and the cut lists of piece k-1 are copied
out.  Files are chunked independently, so the pieces are too.

``HostStreamPipeline`` (and ``chunk_stream_host`` on top of it) chunks one
long stream delivered as host blocks of any size (more than fits on the
device, if need be), resumable block by block.  A chunk depends only on bytes
from its start to start + max_size, so every cut of a prefix except its last
is a cut of the whole stream (Sec. IV: a forced cut at the end of the input is
the only cut the end decides).  Each block is chunked together with the bytes
after the previous block's last proven cut, kept on the device; the copy of a
block to the device overlaps the chunking of the one before; the final cut of
the last block is the stream end.

``HostInPlace`` chunks a batch (or one stream) that stays in pinned host
memory without copying it: the library's kernels read the bytes in place over
the host link, and the chain walk they take loads only the half windows its
scan reaches (Sec. III.B-C leave the rest unread), so a fraction of the input
crosses.  Only the offsets go to the device; the kernels write the cut lists
straight into pinned host memory.

All chunking runs in the library's CUDA kernels; this module moves bytes and
orders streams.
"""
from __future__ import annotations

import collections
from typing import Iterable, Iterator, List, Tuple

import numpy as np

from . import seqcdc


def split_files(offsets: np.ndarray, pieces: int) -> List[Tuple[int, int]]:
    """File ranges [a, b) of about equal bytes; every piece has a file
    (unless there are fewer files than pieces), a file is never split."""
    offs = np.asarray(offsets, dtype=np.int64)
    nfiles = offs.size - 1
    if nfiles <= 0:
        return []
    pieces = max(1, min(pieces, nfiles))
    total = int(offs[-1])
    out, a = [], 0
    for k in range(1, pieces + 1):
        if a >= nfiles:
            break
        target = total * k // pieces
        b = int(np.searchsorted(offs, target, side="left"))
        b = max(a + 1, min(b, nfiles))
        if k == pieces:
            b = nfiles
        out.append((a, b))
        a = b
    return out


class _Slot:
    def __init__(self, torch, dev, p, max_bytes, max_files, tuning):
        self.max_bytes, self.max_files = max_bytes, max_files
        self.cap = max_bytes // p.min_size + max_files
        self.data = torch.empty(max(max_bytes, 16), dtype=torch.uint8, device=dev)
        self.offs = torch.empty(max_files + 1, dtype=torch.int64, device=dev)
        self.cuts = torch.empty(max(self.cap, 1), dtype=torch.int64, device=dev)
        self.co = torch.empty(max_files + 1, dtype=torch.int64, device=dev)
        self.ws_bytes = seqcdc.seqcdc_workspace_size(p, max_bytes, max_files, tuning)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.free = None  # event: the slot's last use is over


class HostBatchPipeline:
    """Reusable pipeline for CSR batches in pinned host memory: device slots,
    streams and pinned staging are kept between calls (they grow when a
    larger piece comes), so a steady stream of batches allocates nothing."""

    def __init__(self, p, tuning=None, device="cuda", slots: int = 3):
        import torch
        self.torch = torch
        self.p, self.tuning, self.nslots = p, tuning, max(1, slots)
        self.dev = torch.device(device)
        self.copy_in = torch.cuda.Stream(self.dev)
        self.compute = torch.cuda.Stream(self.dev)
        self.copy_out = torch.cuda.Stream(self.dev)
        self.pool: List[_Slot] = []
        self.h_cuts, self.h_co, self.h_rel = [], [], []
        self.h_status = None

    def _pinned(self, lst, k, n):
        torch = self.torch
        while len(lst) <= k:
            lst.append(None)
        if lst[k] is None or lst[k].numel() < n:
            lst[k] = torch.empty(max(n, 1), dtype=torch.int64, pin_memory=True)
        return lst[k]

    def _slots(self, max_bytes, max_files, n):
        if any(s.max_bytes < max_bytes or s.max_files < max_files for s in self.pool):
            self.pool = []
        while len(self.pool) < min(self.nslots, n):
            self.pool.append(_Slot(self.torch, self.dev, self.p, max_bytes, max_files,
                                   self.tuning))
        for s in self.pool:
            s.free = None

    def run(self, h_data, h_offsets, pieces: int = 4):
        """(cuts int64, cut_offsets int64) on the host, equal to
        ``chunk_batch`` of the same batch on the device."""
        torch, p, tuning = self.torch, self.p, self.tuning
        offs = np.asarray(h_offsets.numpy() if hasattr(h_offsets, "numpy") else h_offsets,
                          dtype=np.int64)
        nfiles = offs.size - 1
        ranges = split_files(offs, pieces)
        if not ranges:
            return np.empty(0, np.int64), np.zeros(max(nfiles + 1, 1), np.int64)
        self._slots(max(int(offs[b] - offs[a]) for a, b in ranges),
                    max(b - a for a, b in ranges), len(ranges))
        if self.h_status is None or self.h_status.numel() < len(ranges):
            self.h_status = torch.empty(len(ranges), dtype=torch.int32, pin_memory=True)
        caps = []
        for k, (a, b) in enumerate(ranges):
            rel = self._pinned(self.h_rel, k, b - a + 1)
            rel[:b - a + 1].copy_(torch.from_numpy(offs[a:b + 1] - offs[a]))
            caps.append(int(offs[b] - offs[a]) // p.min_size + (b - a))
            self._pinned(self.h_cuts, k, caps[-1])
            self._pinned(self.h_co, k, b - a + 1)
        done = []
        for k, (a, b) in enumerate(ranges):
            s = self.pool[k % len(self.pool)]
            n = int(offs[b] - offs[a])
            if s.free is not None:
                self.copy_in.wait_event(s.free)
            with torch.cuda.stream(self.copy_in):
                s.data[:n].copy_(h_data[int(offs[a]):int(offs[b])], non_blocking=True)
                s.offs[:b - a + 1].copy_(self.h_rel[k][:b - a + 1], non_blocking=True)
                loaded = torch.cuda.Event()
                loaded.record(self.copy_in)
            self.compute.wait_event(loaded)
            cap = caps[k]
            seqcdc.seqcdc_chunk_batch(p, s.data, n, s.offs, b - a, s.cuts, cap, s.co,
                                      s.ws, s.ws_bytes, tuning, self.compute)
            chunked = torch.cuda.Event()
            chunked.record(self.compute)
            self.copy_out.wait_event(chunked)
            with torch.cuda.stream(self.copy_out):
                self.h_co[k][:b - a + 1].copy_(s.co[:b - a + 1], non_blocking=True)
                self.h_cuts[k][:cap].copy_(s.cuts[:cap], non_blocking=True)
                # the piece's device status word (first field of the workspace)
                self.h_status[k:k + 1].copy_(s.ws[:4].view(torch.int32), non_blocking=True)
                s.free = torch.cuda.Event()
                s.free.record(self.copy_out)
            done.append(s.free)
        # Collect in order while the later pieces are still on the GPU: each
        # piece's cuts go into one output array as soon as its copy back is
        # over, so only the last piece's host copy is not overlapped.
        out_cuts = np.empty(max(sum(caps), 1), dtype=np.int64)
        out_co = np.zeros(nfiles + 1, dtype=np.int64)
        base = 0
        for k, (a, b) in enumerate(ranges):
            done[k].synchronize()
            st = int(self.h_status[k])
            if st != seqcdc.SEQCDC_OK:
                for e in done[k + 1:]:   # leave no piece in flight in the slots
                    e.synchronize()
                raise seqcdc.SeqCDCError(st, "chunk_batch_host (device)")
            co = self.h_co[k][:b - a + 1].numpy()
            cnt = int(co[-1])
            out_cuts[base:base + cnt] = self.h_cuts[k][:cnt].numpy()
            out_co[a + 1:b + 1] = co[1:] + base
            base += cnt
        return out_cuts[:base], out_co


def chunk_batch_host(h_data, h_offsets, p, pieces: int = 4, slots: int = 3,
                     tuning=None, device="cuda"):
    """One-off use of ``HostBatchPipeline``: chunk a CSR batch held in pinned
    host memory; returns host (cuts int64, cut_offsets int64)."""
    return HostBatchPipeline(p, tuning, device, slots).run(h_data, h_offsets, pieces)


class HostInPlace:
    """Chunking of input that stays in pinned host memory, read in place by
    the kernels.  Device buffers (offsets, cut lists, workspace) and pinned
    result buffers are kept between calls and grow when a larger call comes,
    so a steady stream of calls allocates nothing."""

    def __init__(self, p, tuning=None, device="cuda"):
        import torch
        self.torch = torch
        self.p, self.tuning = p, tuning
        self.dev = torch.device(device)
        self.stream = torch.cuda.Stream(self.dev)
        self.max_bytes = self.max_files = -1

    def _grow(self, total: int, nfiles: int):
        if total <= self.max_bytes and nfiles <= self.max_files:
            return
        torch, p, dev = self.torch, self.p, self.dev
        self.max_bytes = max(total, self.max_bytes)
        self.max_files = max(nfiles, self.max_files)
        self.cap = self.max_bytes // p.min_size + self.max_files
        self.d_offs = torch.empty(self.max_files + 1, dtype=torch.int64, device=dev)
        self.ws_bytes = seqcdc.seqcdc_workspace_size(p, self.max_bytes, self.max_files,
                                                     self.tuning)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev)
        self.h_offs = torch.empty(self.max_files + 1, dtype=torch.int64, pin_memory=True)
        self.h_co = torch.empty(self.max_files + 1, dtype=torch.int64, pin_memory=True)
        self.h_cuts = torch.empty(max(self.cap, 1), dtype=torch.int64, pin_memory=True)
        self.h_status = torch.empty(1, dtype=torch.int32, pin_memory=True)

    def run(self, h_data, h_offsets):
        """(cuts int64, cut_offsets int64) on the host for a CSR batch whose
        bytes ``h_data`` (a pinned uint8 tensor) stay on the host; equal to
        ``chunk_batch`` of the same batch on the device.  The returned arrays
        are views of buffers the next call reuses."""
        torch = self.torch
        if h_data.dtype != torch.uint8 or h_data.is_cuda or (
                h_data.numel() and not h_data.is_pinned()):
            raise TypeError("HostInPlace.run needs a pinned uint8 host tensor")
        h_data = h_data.view(-1)
        offs = np.asarray(h_offsets.numpy() if hasattr(h_offsets, "numpy") else h_offsets,
                          dtype=np.int64)
        nfiles = offs.size - 1
        total = int(h_data.numel())
        if nfiles < 0 or int(offs[-1]) != total:
            raise ValueError("offsets must end at the byte count")
        self._grow(total, nfiles)
        st = self.stream
        self.h_offs[:nfiles + 1].numpy()[:] = offs
        with torch.cuda.stream(st):
            self.d_offs[:nfiles + 1].copy_(self.h_offs[:nfiles + 1], non_blocking=True)
            # The cut lists and their index are written straight into pinned
            # host memory (mapped, like the input): nothing to copy back.
            seqcdc.seqcdc_chunk_batch(self.p, h_data, total, self.d_offs, nfiles, self.h_cuts,
                                      self.cap, self.h_co, self.ws, self.ws_bytes, self.tuning,
                                      st)
            self.h_status.copy_(self.ws[:4].view(torch.int32), non_blocking=True)
        st.synchronize()
        if int(self.h_status[0]) != 0:
            seqcdc._check(int(self.h_status[0]), "HostInPlace.run (device)")
        n = int(self.h_co[nfiles])
        return self.h_cuts[:n].numpy(), self.h_co[:nfiles + 1].numpy()

    def run_stream(self, h_data):
        """Cut offsets (int64, on the host) of one stream that stays in pinned
        host memory; equal to ``chunk`` of the same bytes on the device."""
        n = int(h_data.numel())
        cuts, _ = self.run(h_data, np.array([0, n], dtype=np.int64))
        return cuts


class HostStreamPipeline:
    """Chunking of one long stream that arrives as host blocks of any size,
    resumable block by block, with the copies overlapped.

    A chunk depends only on the bytes from its start to start + max_size
    (Sec. IV), so every cut of a prefix except its last is a cut of the whole
    stream.  Each block is chunked together with the bytes after the
    previous block's last proven cut (the carried tail, at most max_size
    bytes, kept on the device).  Per block:
      1. its bytes go host -> device into a staging slot on a copy stream
         (``slots`` slots in rotation, reused across calls);
      2. meanwhile the host waits for the previous block's chunking and reads
         its cut count and cut list (small device -> host copies);
      3. on the compute stream the carried tail and the block are copied
         device -> device, back to back, into an aligned work buffer (two in
         rotation), which ``seqcdc_chunk`` chunks; its cut list is copied to
         pinned host memory.
    The copies in run up to ``slots - 1`` blocks ahead of the chunking, so
    the copy engine stays busy while the host does its bookkeeping.  ``feed``
    returns the cuts proven so far that were not returned before (absolute
    offsets; blocks still in flight are not yet chunked); ``finish`` returns
    the rest, ending at the stream end.  Blocks larger than ``block_bytes`` are
    taken in parts.  Pinned host blocks (torch tensors) are copied
    asynchronously; numpy or pageable blocks go through a pinned staging copy
    on the host first.
    """

    def __init__(self, p, tuning=None, device="cuda", block_bytes: int = 128 << 20,
                 slots: int = 3):
        import torch
        self.torch = torch
        self.p, self.tuning = p, tuning
        self.dev = torch.device(device)
        self.B = max(int(block_bytes), 1 << 16)
        self.mx = int(p.max_size)
        self.copy_in = torch.cuda.Stream(self.dev)
        self.compute = torch.cuda.Stream(self.dev)
        n = self.B + self.mx
        self.cap = n // p.min_size + 1
        self.stage = [torch.empty(self.B, dtype=torch.uint8, device=self.dev)
                      for _ in range(max(2, slots))]
        self.h_stage = [None] * len(self.stage)   # pinned staging, made when needed
        self.stage_free = [None] * len(self.stage)
        # a 16-byte aligned work buffer per rotation step (the chunker's rule)
        self.work = [torch.empty(n + 16, dtype=torch.uint8, device=self.dev) for _ in range(2)]
        self.cuts = [torch.empty(self.cap, dtype=torch.int64, device=self.dev) for _ in range(2)]
        self.count = [torch.zeros(1, dtype=torch.int64, device=self.dev) for _ in range(2)]
        self.h_cuts = [torch.empty(self.cap, dtype=torch.int64, pin_memory=True) for _ in range(2)]
        self.h_count = [torch.zeros(1, dtype=torch.int64, pin_memory=True) for _ in range(2)]
        self.ws_bytes = seqcdc.seqcdc_workspace_size(p, n, 1, tuning)
        self.ws = [torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.dev)
                   for _ in range(2)]
        self.h_status = [torch.zeros(1, dtype=torch.int32, pin_memory=True) for _ in range(2)]
        self.reset()

    def reset(self):
        """Start a new stream (the carried tail is dropped)."""
        self.base = 0          # absolute offset of work[cur][0]
        self.nblk = 0          # blocks (parts) chunked so far
        self.nin = 0           # parts copied in so far
        self.inflight = collections.deque()  # parts copied in, not yet chunked
        self.pending = None    # (work index, bytes in the work buffer, event)
        self.carry = (None, 0, 0)  # (work index, offset of the tail, its length)

    def _part(self, blk):
        """Copy one part (<= block_bytes) host -> device staging; returns
        (staging index, length, event)."""
        torch = self.torch
        k = self.nin % len(self.stage)
        self.nin += 1
        n = int(blk.numel() if hasattr(blk, "numel") else blk.size)
        if self.stage_free[k] is not None:
            self.copy_in.wait_event(self.stage_free[k])
        src = blk
        if not (hasattr(blk, "is_pinned") and blk.is_pinned()):
            if self.h_stage[k] is None:
                self.h_stage[k] = torch.empty(self.B, dtype=torch.uint8, pin_memory=True)
            h = self.h_stage[k]
            if self.stage_free[k] is not None:
                self.stage_free[k].synchronize()  # its last copy out of h_stage is over
            h[:n].copy_(torch.from_numpy(np.ascontiguousarray(blk, dtype=np.uint8))
                        if not hasattr(blk, "numel") else blk)
            src = h[:n]
        with torch.cuda.stream(self.copy_in):
            self.stage[k][:n].copy_(src, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.copy_in)
        return k, n, ev

    def _collect(self, final: bool):
        """Wait for the pending chunking; return its proven cuts (all of them
        when `final`) and set the carried tail."""
        if self.pending is None:
            return np.empty(0, np.int64)
        w, nbytes, ev = self.pending
        self.pending = None
        ev.synchronize()
        st = int(self.h_status[w][0])
        if st != seqcdc.SEQCDC_OK:
            raise seqcdc.SeqCDCError(st, "HostStreamPipeline (device)")
        k = int(self.h_count[w][0])
        cuts = self.h_cuts[w][:k].numpy()
        if final or k <= 1:
            keep = cuts if final else cuts[:0]
        else:
            keep = cuts[:-1]
        last = int(keep[-1]) if keep.size and not final else 0
        out = keep + self.base
        if not final:
            self.carry = (w, last, nbytes - last)
            self.base += last
        return out

    def _chunk_part(self, k, n, loaded):
        torch = self.torch
        w = self.nblk % 2
        cw, coff, clen = self.carry
        self.compute.wait_event(loaded)
        with torch.cuda.stream(self.compute):
            if clen:
                self.work[w][:clen].copy_(self.work[cw][coff:coff + clen])
            self.work[w][clen:clen + n].copy_(self.stage[k][:n])
            freed = torch.cuda.Event()
            freed.record(self.compute)
        self.stage_free[k] = freed
        total = clen + n
        seqcdc.seqcdc_chunk(self.p, self.work[w], total, self.cuts[w], self.cap, self.count[w],
                            self.ws[w], self.ws_bytes, self.tuning, self.compute)
        with torch.cuda.stream(self.compute):
            self.h_count[w].copy_(self.count[w], non_blocking=True)
            self.h_cuts[w][:self.cap].copy_(self.cuts[w], non_blocking=True)
            self.h_status[w].copy_(self.ws[w][:4].view(torch.int32), non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.compute)
        self.pending = (w, total, ev)
        self.nblk += 1

    def feed(self, blk) -> np.ndarray:
        """Add a block (pinned torch uint8 tensor, or numpy bytes); returns the
        cuts proven so far that were not returned before (absolute)."""
        outs = []
        n = int(blk.numel() if hasattr(blk, "numel") else np.asarray(blk).size)
        for a in range(0, n, self.B):
            self.inflight.append(self._part(blk[a:min(n, a + self.B)]))
            # chunk the oldest part once the copies ahead fill the free slots
            while len(self.inflight) >= len(self.stage):
                outs.append(self._advance())
        return np.concatenate(outs) if outs else np.empty(0, np.int64)

    def _advance(self) -> np.ndarray:
        """Chunk the oldest part copied in: wait for the part before it,
        then enqueue it; returns the cuts the wait proved."""
        k, m, loaded = self.inflight.popleft()
        out = self._collect(final=False)
        self._chunk_part(k, m, loaded)
        return out

    def finish(self) -> np.ndarray:
        """The remaining cuts, the last one at the stream end; then reset."""
        outs = []
        while self.inflight:
            outs.append(self._advance())
        outs.append(self._collect(final=True))   # the last part is pending
        self.reset()
        return np.concatenate(outs)

    def run(self, blocks) -> np.ndarray:
        """Cut list of the whole stream given as an iterable of blocks."""
        parts = [self.feed(b) for b in blocks]
        parts.append(self.finish())
        return np.concatenate(parts)


def chunk_stream_host(blocks: Iterable[np.ndarray], p, tuning=None,
                      device="cuda", block_bytes: int = 128 << 20) -> Iterator[np.ndarray]:
    """Chunk one stream given as host blocks (any sizes); yields the absolute
    cut offsets block by block (their concatenation is the stream's cut
    list), through a HostStreamPipeline (copies overlapped with chunking)."""
    pipe = HostStreamPipeline(p, tuning, device, block_bytes)
    for blk in blocks:
        out = pipe.feed(blk)
        if out.size:
            yield out
    out = pipe.finish()
    if out.size:
        yield out
