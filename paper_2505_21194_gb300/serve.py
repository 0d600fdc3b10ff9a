"""Continuous-batching chunking server.

Requests are byte strings held in pinned host memory that arrive over time
(open loop).  The server admits arrived requests first come, first served,
while the request bytes in flight on the device stay within an HBM budget.
Each admission round becomes one CSR batch: the requests are copied into one
device buffer on a copy stream, chunked by ``seqcdc_chunk_batch`` on a compute
stream (each file of a batch is chunked as if it were alone), and their cut
lists are copied back to pinned host memory.  A request's latency runs from
its arrival to the completion of its batch, read on the device clock (CUDA
events) and aligned to the host clock at the start of the run.

The batching rule (``form_batch``) and the statistics are plain functions so
that they can be checked without a GPU.  The chunking itself runs only in the
library's CUDA kernels.
"""
from __future__ import annotations

import collections
import dataclasses
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
class _Batch:
    reqs: List[Request]
    nbytes: int
    done: object          # torch.cuda.Event after the copy back
    keep: tuple           # device tensors alive until the batch is done
    h_cuts: object        # pinned host int64
    h_co: object          # pinned host int64
    slot: int             # staging slot


@dataclasses.dataclass
class ServeStats:
    requests: int
    batches: int
    bytes: int
    wall_s: float
    sustained_gbs: float
    latency: Dict[str, float]
    results: Dict[int, np.ndarray]      # cut lists of the requests asked for


class Server:
    """One GPU, one copy stream and one compute stream; up to ``max_inflight``
    batches in the pipeline (copy of one overlapping the chunking of the
    previous)."""

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
        # Pinned staging for each pipeline slot, allocated once: offsets in,
        # cut lists and CSR index out (a batch's cut list is bounded by its
        # bytes / min_size + its files).
        big = max(self.max_batch, int(self.sizes.max(initial=0)))
        cap = big // p.min_size + self.max_files
        self._stage = [(torch.empty(self.max_files + 1, dtype=torch.int64, pin_memory=True),
                        torch.empty(cap, dtype=torch.int64, pin_memory=True),
                        torch.empty(self.max_files + 1, dtype=torch.int64, pin_memory=True))
                       for _ in range(self.max_inflight)]
        self._free_stage = list(range(self.max_inflight))

    # -- one batch ---------------------------------------------------------
    def _launch(self, reqs: List[Request]) -> _Batch:
        torch = self.torch
        sizes = np.array([r.nbytes for r in reqs], dtype=np.int64)
        offs = np.zeros(len(reqs) + 1, dtype=np.int64)
        np.cumsum(sizes, out=offs[1:])
        total = int(offs[-1])
        nfiles = len(reqs)
        cap = total // self.p.min_size + nfiles
        slot = self._free_stage.pop()
        h_offs_all, h_cuts_all, h_co_all = self._stage[slot]
        h_offs = h_offs_all[:nfiles + 1]
        h_offs.copy_(torch.from_numpy(offs))
        with torch.cuda.stream(self.copy):
            d_data = torch.empty(max(total, 16), dtype=torch.uint8, device=self.device)
            for r, o in zip(reqs, offs[:-1].tolist()):
                src = self.pool[int(self.offs[r.payload]):int(self.offs[r.payload + 1])]
                d_data[o:o + r.nbytes].copy_(src, non_blocking=True)
            d_offs = h_offs.to(self.device, non_blocking=True)
            copied = torch.cuda.Event()
            copied.record(self.copy)
        self.compute.wait_event(copied)
        with torch.cuda.stream(self.compute):
            d_cuts = torch.empty(max(cap, 1), dtype=torch.int64, device=self.device)
            d_co = torch.empty(nfiles + 1, dtype=torch.int64, device=self.device)
            ws_bytes = seqcdc.seqcdc_workspace_size(self.p, total, nfiles, self.tuning)
            d_ws = torch.empty(ws_bytes, dtype=torch.uint8, device=self.device)
            # the copy stream wrote these; the compute stream reads them
            d_data.record_stream(self.compute)
            d_offs.record_stream(self.compute)
            seqcdc.seqcdc_chunk_batch(self.p, d_data, total, d_offs, nfiles, d_cuts,
                                      cap, d_co, d_ws, ws_bytes, self.tuning,
                                      self.compute)
            h_cuts = h_cuts_all[:max(cap, 1)]
            h_co = h_co_all[:nfiles + 1]
            h_cuts.copy_(d_cuts, non_blocking=True)
            h_co.copy_(d_co, non_blocking=True)
            done = torch.cuda.Event(enable_timing=True)
            done.record(self.compute)
        return _Batch(reqs, total, done, (d_data, d_offs, d_cuts, d_co, d_ws, h_offs),
                      h_cuts, h_co, slot)

    # -- the serving loop --------------------------------------------------
    def run(self, arrivals: Iterable[Request], keep: Optional[set] = None,
            poll_s: float = 50e-6) -> ServeStats:
        torch = self.torch
        arrivals = sorted(arrivals, key=lambda r: r.arrival)
        keep = keep or set()
        queue: collections.deque = collections.deque()
        inflight: collections.deque = collections.deque()
        inflight_bytes = 0
        lat, results = [], {}
        nbatches, nbytes = 0, 0
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
            progressed = False
            while inflight and inflight[0].done.query():
                b = inflight.popleft()
                t_done = start.elapsed_time(b.done) / 1e3
                last_done = max(last_done, t_done)
                co = b.h_co.numpy()
                cuts = b.h_cuts.numpy()
                for j, r in enumerate(b.reqs):
                    lat.append(t_done - r.arrival)
                    if r.rid in keep:
                        results[r.rid] = cuts[co[j]:co[j + 1]].copy()
                inflight_bytes -= b.nbytes
                nbytes += b.nbytes
                self._free_stage.append(b.slot)
                progressed = True
            if queue and len(inflight) < self.max_inflight:
                k = form_batch(queue, inflight_bytes, self.budget, self.max_batch,
                               self.max_files)
                if k:
                    reqs = [queue.popleft() for _ in range(k)]
                    b = self._launch(reqs)
                    inflight.append(b)
                    inflight_bytes += b.nbytes
                    nbatches += 1
                    progressed = True
            if not progressed:
                time.sleep(poll_s)
        wall = max(last_done - first_arrival, 1e-9)
        return ServeStats(len(lat), nbatches, nbytes, wall, nbytes / wall / 1e9,
                          latency_stats(lat), results)
