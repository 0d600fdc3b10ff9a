"""Continuous-batching chunking server.

Requests are byte strings held in pinned host memory that arrive over time
(open loop).  The server admits arrived requests first come, first served,
while the request bytes in flight on the device stay within an HBM budget.
Each admission round becomes one CSR batch in one of a few preallocated
pipeline slots (device buffers for the bytes, offsets, cut lists and a
workspace that fits any batch on either chunking path), so that serving
allocates no device memory per batch: the requests are copied into the slot
on a copy stream and chunked by ``seqcdc_chunk_batch`` on a compute stream
(each file of a batch is chunked as if it were alone).  Cut lists stay on the
device; only the batch's 4-byte status word comes back, and the cut lists of
the requests the caller asks for are kept as device tensors.  A request's
latency runs from its arrival to the completion of its batch's chunking, read
on the device clock (CUDA events) and aligned to the host clock at the start
of the run.

The batching rule (``form_batch``) and the statistics are plain functions so
that they can be checked without a GPU.  The chunking itself runs only in the
library's CUDA kernels.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import time
from typing import Dict, Iterable, List, Optional, Sequence

import numpy as np

from . import seqcdc

GIB = 1 << 30


@dataclasses.dataclass
class Request:
    rid: int
    payload: int       # index of the payload in the server's pool
    nbytes: int
    arrival: float     # seconds from the start of the run


def form_batch(queue: Sequence[Request], inflight_bytes: int, budget: int,
               max_batch_bytes: int, max_files: int = 1 << 30) -> int:
    """How many requests at the head of ``queue`` form the next batch.

    First come, first served: requests are taken in order while the batch
    stays within ``max_batch_bytes`` (a request larger than that forms a batch
    alone) and ``max_files`` requests, and the bytes in flight stay within
    ``budget``.  The head request is never skipped, so the order of
    completion follows the order of arrival batch by batch.
    """
    take, total = 0, 0
    for r in queue:
        if take and (total + r.nbytes > max_batch_bytes or take >= max_files):
            break
        if inflight_bytes + total + r.nbytes > budget:
            break
        take += 1
        total += r.nbytes
    return take


def withdraw(queue, withdrawn) -> int:
    """Remove from ``queue`` (a deque of requests; in place, order kept)
    every request whose id is in ``withdrawn``; return how many went."""
    stay = [r for r in queue if r.rid not in withdrawn]
    gone = len(queue) - len(stay)
    if gone:
        queue.clear()
        queue.extend(stay)
    return gone


class Cancellations:
    """Client cancellations of a run: request id -> the time (seconds from
    the start, like arrivals) at which the client withdraws the request.

    ``tick(now, queue, narrived)`` is called by the serving loop after the
    arrivals up to ``now`` (``narrived`` of them so far) have joined
    ``queue``: every request whose cancellation time has come and that is
    still queued, or arrives later, is removed before admission.  A request
    admitted before its cancellation runs to completion; ``too_late`` counts
    those."""

    def __init__(self, cancels: Optional[Dict[int, float]] = None):
        self.at = sorted((float(t), int(rid)) for rid, t in (cancels or {}).items())
        self.rids = {rid for _, rid in self.at}
        self.withdrawn: set = set()
        self.next = self.seen = self.cancelled = 0

    def __bool__(self) -> bool:
        return bool(self.at)

    def tick(self, now: float, queue, narrived: int) -> None:
        grew = False
        while self.next < len(self.at) and self.at[self.next][0] <= now:
            self.withdrawn.add(self.at[self.next][1])
            self.next += 1
            grew = True
        if self.withdrawn and (grew or narrived > self.seen):
            self.cancelled += withdraw(queue, self.withdrawn)
        self.seen = narrived

    def too_late(self, arrivals: Sequence[Request]) -> int:
        return sum(1 for r in arrivals if r.rid in self.rids) - self.cancelled


def latency_stats(lat_s: Sequence[float]) -> Dict[str, float]:
    """p50 / p99 / mean / max of latencies given in seconds, in milliseconds."""
    a = np.asarray(lat_s, dtype=np.float64) * 1e3
    if a.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None, "max_ms": None}
    return {"p50_ms": float(np.percentile(a, 50)), "p99_ms": float(np.percentile(a, 99)),
            "mean_ms": float(a.mean()), "max_ms": float(a.max())}


def poisson_arrivals(rate_per_s: float, duration_s: float, npayloads: int,
                     sizes: Sequence[int], seed: int) -> List[Request]:
    """Open-loop arrivals: exponential gaps at ``rate_per_s`` over
    ``duration_s``; each request names a payload drawn uniformly."""
    rng = np.random.default_rng(seed)
    out, t, rid = [], 0.0, 0
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t > duration_s:
            return out
        k = int(rng.integers(npayloads))
        out.append(Request(rid, k, int(sizes[k]), t))
        rid += 1


@dataclasses.dataclass
class _Slot:
    """Device buffers of one pipeline slot, allocated once: request bytes,
    CSR offsets, cut lists, CSR index and a workspace that fits any batch of
    up to max_bytes bytes and max_files files on either chunking path."""
    data: object
    offs: object
    cuts: object
    co: object
    ws: object
    ws_bytes: int
    h_offs: object        # pinned staging for the offsets
    h_status: object      # pinned: the device status word of the slot's last batch
    h_co: object          # pinned: the CSR index of the slot's last batch with kept requests


@dataclasses.dataclass
class _Batch:
    reqs: List[Request]
    nbytes: int
    done: object          # CUDA event: the batch is chunked (latency ends here)
    ready: object         # CUDA event: its status word (and kept results) copied
    slot: int
    kept: Optional[List[int]]  # places in the batch of the requests whose cuts are kept


@dataclasses.dataclass
class ServeStats:
    requests: int
    batches: int
    bytes: int
    wall_s: float
    sustained_gbs: float
    latency: Dict[str, float]
    results: Dict[int, object]      # cut lists (device tensors) of the requests asked for
    cancelled: int = 0              # requests withdrawn before admission (never chunked)
    cancel_too_late: int = 0        # cancellations that came after admission (served)


class Server:
    """One GPU, one copy stream and one compute stream; up to ``max_inflight``
    batches in the pipeline (the copy of one overlapping the chunking of the
    previous), each in its own preallocated slot, so that serving allocates
    no device memory per batch."""

    def __init__(self, p, pool, pool_offsets, budget_bytes: int = 64 * GIB,
                 max_batch_bytes: int = 4 * GIB, max_inflight: int = 3,
                 tuning=None, device: str = "cuda", max_batch_files: int = 4096):
        import torch
        if not pool.is_pinned():
            raise ValueError("the payload pool must be pinned host memory")
        self.torch = torch
        self.p = p
        self.pool = pool
        self.offs = np.asarray(pool_offsets, dtype=np.int64)
        self.sizes = np.diff(self.offs)
        if self.sizes.max(initial=0) > budget_bytes:
            raise ValueError("a payload is larger than the HBM budget")
        self.budget = int(budget_bytes)
        self.max_batch = int(max_batch_bytes)
        self.max_inflight = int(max_inflight)
        self.tuning = tuning
        self.device = torch.device(device)
        self.copy = torch.cuda.Stream(self.device)
        self.compute = torch.cuda.Stream(self.device)
        self.max_files = int(max_batch_files)
        seqcdc.load_library()
        # A batch holds at most max_batch bytes, or one payload larger than that.
        big = max(self.max_batch, int(self.sizes.max(initial=0)), 16)
        cap = big // p.min_size + self.max_files
        nf = self.max_files
        ws_bytes = max(seqcdc.seqcdc_workspace_size(p, big, nf, (0, 0, seqcdc.ALGO_MAP, 0)),
                       seqcdc.seqcdc_workspace_size(p, big, nf, (0, 0, seqcdc.ALGO_WALK, 0)))
        if tuning is not None:
            ws_bytes = max(ws_bytes, seqcdc.seqcdc_workspace_size(p, big, nf, tuning))
        dev = self.device
        self._slots = [_Slot(torch.empty(big, dtype=torch.uint8, device=dev),
                             torch.empty(nf + 1, dtype=torch.int64, device=dev),
                             torch.empty(cap, dtype=torch.int64, device=dev),
                             torch.empty(nf + 1, dtype=torch.int64, device=dev),
                             torch.empty(ws_bytes, dtype=torch.uint8, device=dev), ws_bytes,
                             torch.empty(nf + 1, dtype=torch.int64, pin_memory=True),
                             torch.zeros(1, dtype=torch.int32, pin_memory=True),
                             torch.empty(nf + 1, dtype=torch.int64, pin_memory=True))
                       for _ in range(self.max_inflight)]
        self._free = list(range(self.max_inflight))

    # -- one batch ---------------------------------------------------------
    def _launch(self, reqs: List[Request], keep: set) -> _Batch:
        torch = self.torch
        sizes = np.array([r.nbytes for r in reqs], dtype=np.int64)
        offs = np.zeros(len(reqs) + 1, dtype=np.int64)
        np.cumsum(sizes, out=offs[1:])
        total, nfiles = int(offs[-1]), len(reqs)
        cap = total // self.p.min_size + nfiles
        k = self._free.pop()
        s = self._slots[k]
        # The slot's previous batch has completed (it was popped as done), so
        # its staging and device buffers are free.
        s.h_offs[:nfiles + 1].copy_(torch.from_numpy(offs))
        src_off = self.offs[np.fromiter((r.payload for r in reqs), dtype=np.int64,
                                        count=nfiles)]
        with torch.cuda.stream(self.copy):
            # every request's bytes into the slot, one async copy each,
            # enqueued by the library in one call
            seqcdc.seqcdc_copy_ranges(s.data, self.pool, offs[:-1], src_off, sizes, self.copy)
            s.offs[:nfiles + 1].copy_(s.h_offs[:nfiles + 1], non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(self.copy)
        self.compute.wait_event(copied)
        seqcdc.seqcdc_chunk_batch(self.p, s.data, total, s.offs, nfiles, s.cuts, cap, s.co,
                                  s.ws, s.ws_bytes, self.tuning, self.compute)
        with torch.cuda.stream(self.compute):
            done = torch.cuda.Event(enable_timing=True)
            done.record(self.compute)
            # the batch's device status word (4 bytes back per batch)
            s.h_status.copy_(s.ws[:4].view(torch.int32), non_blocking=True)
            kept = [j for j, r in enumerate(reqs) if r.rid in keep] or None
            if kept is not None:
                # the batch's CSR index comes back with the status word, so
                # that taking the kept cut lists needs no synchronisation
                s.h_co[:nfiles + 1].copy_(s.co[:nfiles + 1], non_blocking=True)
            ready = torch.cuda.Event()
            ready.record(self.compute)
        return _Batch(reqs, total, done, ready, k, kept)

    # -- the serving loop --------------------------------------------------
    def run(self, arrivals: Iterable[Request], keep: Optional[set] = None,
            poll_s: float = 0.0, cancels: Optional[Dict[int, float]] = None) -> ServeStats:
        """Serve ``arrivals``; keep the cut lists of the request ids in
        ``keep``.  ``cancels`` maps request ids to the time (seconds from the
        start, like arrivals) at which their client withdraws them: a request
        still queued then (or not yet arrived) is dropped without being
        chunked; one already admitted runs to completion, and the
        cancellation is counted as too late."""
        # The Python garbage collector is held off while serving: a full
        # collection in a process with many live objects pauses the
        # admission loop for tens to hundreds of milliseconds.
        was_enabled = gc.isenabled()
        gc.collect()
        gc.disable()
        try:
            return self._run(arrivals, keep, poll_s, cancels)
        finally:
            if was_enabled:
                gc.enable()

    def _run(self, arrivals, keep, poll_s, cancels=None) -> ServeStats:
        torch = self.torch
        arrivals = sorted(arrivals, key=lambda r: r.arrival)
        keep = keep or set()
        queue: collections.deque = collections.deque()
        inflight: collections.deque = collections.deque()
        inflight_bytes = 0
        lat, results = [], {}
        nbatches, nbytes = 0, 0
        # The cut lists the caller asks for stay on the device, in one buffer
        # sized here for the requests kept (a request of n bytes has at most
        # n / min_size + 1 cuts), so that the loop itself allocates nothing.
        kept_cap = sum(r.nbytes // self.p.min_size + 1 for r in arrivals if r.rid in keep)
        kept_buf = (torch.empty(kept_cap, dtype=torch.int64, device=self.device)
                    if kept_cap else None)
        kept_used = 0
        cancel = Cancellations(cancels)
        cancelling = bool(cancel)
        first_arrival = arrivals[0].arrival if arrivals else 0.0
        last_done = first_arrival
        torch.cuda.synchronize(self.device)
        start = torch.cuda.Event(enable_timing=True)
        start.record(self.compute)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        i = 0
        while i < len(arrivals) or queue or inflight:
            now = time.perf_counter() - t0
            while i < len(arrivals) and arrivals[i].arrival <= now:
                queue.append(arrivals[i])
                i += 1
            if cancelling:
                cancel.tick(now, queue, i)
            progressed = False
            while inflight and inflight[0].ready.query():
                b = inflight.popleft()
                t_done = start.elapsed_time(b.done) / 1e3
                last_done = max(last_done, t_done)
                for r in b.reqs:
                    lat.append(t_done - r.arrival)
                st = int(self._slots[b.slot].h_status[0])
                if st != seqcdc.SEQCDC_OK:
                    raise seqcdc.SeqCDCError(st, "serve batch (device)")
                if b.kept is not None:
                    # copy the kept requests' cuts out of the slot before it
                    # is reused (its next chunking is ordered after, on the
                    # same stream)
                    s = self._slots[b.slot]
                    co_h = s.h_co[:len(b.reqs) + 1].numpy()  # written before `ready`
                    with torch.cuda.stream(self.compute):
                        for j in b.kept:
                            a, e = int(co_h[j]), int(co_h[j + 1])
                            dst = kept_buf[kept_used:kept_used + (e - a)]
                            dst.copy_(s.cuts[a:e], non_blocking=True)
                            results[b.reqs[j].rid] = dst
                            kept_used += e - a
                inflight_bytes -= b.nbytes
                nbytes += b.nbytes
                self._free.append(b.slot)
                progressed = True
            if queue and len(inflight) < self.max_inflight and self._free:
                k = form_batch(queue, inflight_bytes, self.budget, self.max_batch,
                               self.max_files)
                if k:
                    reqs = [queue.popleft() for _ in range(k)]
                    b = self._launch(reqs, keep)
                    inflight.append(b)
                    inflight_bytes += b.nbytes
                    nbatches += 1
                    progressed = True
            if not progressed and poll_s > 0:
                # (the default spins: a sleeping loop wakes up late on a busy
                # host, and every wake-up is a request's latency)
                time.sleep(poll_s)
        torch.cuda.synchronize(self.device)
        wall = max(last_done - first_arrival, 1e-9)
        return ServeStats(len(lat), nbatches, nbytes, wall, nbytes / wall / 1e9,
                          latency_stats(lat), results, cancel.cancelled,
                          cancel.too_late(arrivals))
