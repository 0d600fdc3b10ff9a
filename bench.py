"""Benchmark: chunked GB/s of the SeqCDC CUDA chunker on GB300.

Workload (one "step" = one pass of the whole chunking path over one batch):
10,000 files with log-normal sizes (median 256 KiB, sigma 1.5, clamped to
4 KiB..64 MiB, ~7.2 GiB in all), half uniform random / half order-1 Markov
text content in 64 KiB pieces, laid out in CSR; 8 KiB parameter setting,
increasing mode.  Inputs are generated on the host from a fixed seed, copied
to HBM once, and are far larger than L2 (no flush needed between steps).

Printed: a `detail:` line with the verbose results, then the one JSON line.
The JSON line carries the metric, the device-resident throughput (`value`:
the K timed steps as one CUDA graph, on the path the autotuner picks: the
chain walk for this batch), the end-to-end throughput through host buffers
(`e2e`), the roofline of the dominant kernel (with the path and its sizes),
clocks, the CPU oracle as a reported baseline, and flat scalar fields for
the rest: the same steps launched directly, the plain one-launch-per-file
loop and the other path on the same batch; the single streams (16 MiB
random, the 1 GiB backup-like stream, the 64 GiB adversarial stream) as a
graph and as direct calls, with their path and kernel roofline fraction; p50/p99 latency and
sustained GB/s of the continuous-batching server under open-loop Poisson
arrivals at 25, 50, 100 and 200 GB/s offered load; the deduplication savings
of the backup-like stream; SHA-256 fingerprinting; the mean chunk sizes of
the parameter sweep.  `config` is the same dict in both arms.

`--impl reference` times the CPU oracle (the plain single-threaded chunker,
files spread over the host cores) on the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "chunked GB/s on 1 GB300 vs HBM roofline (batched vs plain); p50/p99 serve latency"
NFILES = 10000
SEED = 0
KIB = 8
MODE = 0


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling in the background (read-only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self, t0: float, t1: float):
        rows = []
        for t, line in self.samples:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((t, parts))
        inside = [r for r in rows if t0 <= r[0] <= t1]
        if not inside and rows:  # region shorter than the sampling period
            inside = sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:3]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"],
                    "samples": 0}
        sm = [float(p[1]) for _, p in inside if p[1].replace(".", "").isdigit()]
        mx = [float(p[2]) for _, p in inside if p[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, p in inside:
            for name, v in zip(names, p[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(inside)}


def bind_to_gpu_numa(gpu_index: int):
    """Run this process on the CPUs local to the GPU (the GPU's PCI device
    lists them in sysfs), so that pinned host buffers are allocated in memory
    next to it: host<->device copies from the other socket's memory are much
    slower.  Returns the CPUs bound to, or None when unknown."""
    try:
        bus = subprocess.run(["nvidia-smi", "--query-gpu=pci.bus_id", "--format=csv,noheader",
                              "-i", str(gpu_index)], capture_output=True, text=True,
                             timeout=30).stdout.strip().lower()
        dom, rest = bus.split(":", 1)
        path = "/sys/bus/pci/devices/%s:%s/local_cpulist" % (dom[-4:], rest)
        cpus = set()
        with open(path) as f:
            for part in f.read().strip().split(","):
                if "-" in part:
                    a, b = part.split("-")
                    cpus.update(range(int(a), int(b) + 1))
                elif part:
                    cpus.add(int(part))
        cpus &= set(os.sched_getaffinity(0))
        if cpus:
            os.sched_setaffinity(0, cpus)
            return sorted(cpus)
    except Exception:
        pass
    return None


def max_over_ranks(x: float, device) -> float:
    """The largest value of x over all ranks (the job is as slow as its
    slowest rank); x itself without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(rank: int, nfiles: int = NFILES):
    from paper_2505_21194_gb300 import workloads as W
    return W.file_batch(nfiles, seed=SEED + rank)


def workload_config(total: int, nfiles: int) -> dict:
    """The workload both arms report (the same dict, so that the two lines
    describe the same configuration)."""
    return {"workload": "batched: %d log-normal files (median 256 KiB, sigma 1.5, "
                        "4 KiB..64 MiB), half random / half Markov text, CSR" % nfiles,
            "setting": "8 KiB (Table I; min 4 KiB, max 16 KiB)", "mode": "increasing",
            "total_bytes": int(total), "nfiles": int(nfiles),
            "l2": "inputs (%.1f GiB) far larger than L2; no flush" % (total / 2**30)}


# Source files each dominant kernel is built from: a DRAM-traffic record
# under profiles/ is used only while the hash of their code (comments
# removed) still matches.
KERNEL_SOURCES = {
    "walk_kernel": ("paper_2505_21194_gb300/csrc/walk.cu",
                    "paper_2505_21194_gb300/csrc/common.cuh"),
    "map_kernel": ("paper_2505_21194_gb300/csrc/seqcdc.cu",
                   "paper_2505_21194_gb300/csrc/common.cuh"),
}


def _traffic_record(kernel: str):
    """DRAM bytes per unit from the committed ncu summary, if still current."""
    path = os.path.join(ROOT, "profiles", "%s_traffic.json" % kernel)
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    return d if d.get("source_sha256") == _source_hash(kernel) else None


def _strip_comments(src: str) -> str:
    """C/C++ source without its comments and blank lines: the code a traffic
    record was measured on, unaffected by edits to comments alone."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c == '"' or c == "'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = [l.rstrip() for l in "".join(out).splitlines()]
    return "\n".join(l for l in lines if l)


def _source_hash(kernel: str):
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            h.update(_strip_comments(f.read()).encode())
    return h.hexdigest()


def scan_span_bytes(d_cuts, d_co, ncuts, p):
    """Bytes the chunk chain scans: for every chunk, from its scan start
    (min_size - SeqLength bytes in, Sec. III.B) to its end."""
    import torch
    cuts = d_cuts[:ncuts]
    starts = torch.zeros_like(cuts)
    if ncuts > 1:
        starts[1:] = cuts[:-1]
    first = d_co[:-1][d_co[:-1] < d_co[1:]]  # first cut of every non-empty file
    starts[first] = 0
    skip = max(int(p.min_size) - int(p.seq_length), 0)
    return int(torch.clamp(cuts - starts - skip, min=0).sum().item())


def cpu_oracle_pass(data, offs, threads):
    import oracle
    p = oracle.presets(KIB, MODE)
    t = time.perf_counter()
    cuts, _ = oracle.chunk_batch_threaded(data, offs, p, threads)
    return time.perf_counter() - t, cuts.size


def run_reference(args):
    rank, world, _ = _dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    data, offs = make_workload(0, args.nfiles)
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpu_oracle_pass(data, offs, threads)
    total = 0.0
    for _ in range(args.steps):
        dt, _ = cpu_oracle_pass(data, offs, threads)
        total += dt
    gbs = data.size * args.steps / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gbs, 3), "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": workload_config(data.size, offs.size - 1),
        "cpu_baseline": {"value": round(gbs, 3), "unit": "GB/s", "cores": threads,
                         "kind": "oracle",
                         "sample": "full 10,000-file batch per step, files spread over %d "
                                   "host threads, single-threaded chunker per file" % threads},
        "e2e": {"value": round(gbs, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def run_gpu(args):
    import torch

    from paper_2505_21194_gb300 import seqcdc

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    numa_cpus = bind_to_gpu_numa(dev.index)
    seqcdc.load_library()

    data_np, offs_np = make_workload(rank, args.nfiles)
    total = int(data_np.size)
    nfiles = offs_np.size - 1
    p = seqcdc.seqcdc_params(KIB, MODE)
    d_data = torch.from_numpy(data_np).to(dev)
    d_offs = torch.from_numpy(offs_np.astype(np.int64)).to(dev)
    tune_src = "library default"
    algos = {"auto": seqcdc.ALGO_AUTO, "map": seqcdc.ALGO_MAP, "walk": seqcdc.ALGO_WALK}
    if args.segment_bytes or args.threads or args.algorithm != "auto" or args.piece_bytes:
        best = (args.segment_bytes, args.threads, algos[args.algorithm], args.piece_bytes)
        tune_src = "command line"
    elif not args.no_autotune:
        # Path and sizes from the autotuner, timed on this device-resident
        # batch (cached per GPU model / parameters / workload shape).
        from paper_2505_21194_gb300 import autotune
        best = autotune.autotune(p, d_data, d_offs)
        tune_src = "autotuned on this batch"
        torch.cuda.empty_cache()  # the candidates' workspaces
    else:
        best = (0, 0, seqcdc.ALGO_AUTO, 0)
    tuning = seqcdc.Tuning(*best)
    eff = seqcdc.seqcdc_resolve_tuning(p, tuning)
    walk = seqcdc.seqcdc_algorithm(p, total, nfiles, True, 1 << 62, tuning) == seqcdc.ALGO_WALK
    cap = total // p.min_size + nfiles
    ws_bytes = seqcdc.seqcdc_workspace_size(p, total, nfiles, tuning)

    d_cuts = torch.empty(cap, dtype=torch.int64, device=dev)
    d_co = torch.empty(nfiles + 1, dtype=torch.int64, device=dev)
    d_ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(st=None):
        seqcdc.seqcdc_chunk_batch(p, d_data, total, d_offs, nfiles, d_cuts, cap,
                                  d_co, d_ws, ws_bytes, tuning, st or stream)

    for _ in range(max(args.warmup, 1)):
        step()
    st = seqcdc.seqcdc_status(d_ws, stream)
    if st != 0:
        raise RuntimeError("device status %d during warm-up" % st)
    ncuts = int(d_co[-1].item())
    path_stats = seqcdc.seqcdc_stats(d_ws, stream, walk=walk)

    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    time.sleep(0.3)
    kb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ke = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    for e in kb + ke:  # torch creates the CUDA event on its first record
        e.record(stream)
    # The timed steps run as one CUDA graph holding exactly K steps (the
    # batched form is launched as a graph); each step's dominant kernel is
    # bracketed by its own pair of events, recorded on every replay.
    graph = None
    if not args.no_graph:
        gs = torch.cuda.Stream(dev)
        gs.wait_stream(stream)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(gs):
            step(gs)  # untimed, on the capture stream
            gs.synchronize()
            with torch.cuda.graph(graph, stream=gs):
                for i in range(args.steps):
                    seqcdc.seqcdc_profile_events(kb[i], ke[i])
                    step(gs)
            seqcdc.seqcdc_profile_events(None, None)
        stream.wait_stream(gs)
        graph.replay()  # an untimed launch of the graph itself
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.time()
    t_begin.record(stream)
    if graph is not None:
        graph.replay()
    else:
        for i in range(args.steps):
            seqcdc.seqcdc_profile_events(kb[i], ke[i])
            step()
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    wall1 = time.time()
    seqcdc.seqcdc_profile_events(None, None)
    if world > 1:
        torch.distributed.barrier()
    time.sleep(0.25)
    sampler.stop()
    clocks = sampler.summary(wall0, wall1)
    st = seqcdc.seqcdc_status(d_ws, stream)
    if st != 0:
        raise RuntimeError("device status %d in the timed region" % st)
    ms_step = t_begin.elapsed_time(t_end) / args.steps
    seg_ms = sum(kb[i].elapsed_time(ke[i]) for i in range(args.steps)) / args.steps
    if world > 1:
        ms_step = max_over_ranks(ms_step, dev)
    gbs = total * world / (ms_step * 1e-3) / 1e9

    # End to end through host buffers: H2D of the batch, chunking, D2H of the
    # CSR index and the cut list, every step.
    h_data = torch.from_numpy(data_np).pin_memory()
    h_offs = torch.from_numpy(offs_np.astype(np.int64)).pin_memory()
    h_co = torch.empty(nfiles + 1, dtype=torch.int64).pin_memory()
    h_cuts = torch.empty(cap, dtype=torch.int64).pin_memory()
    e2e_steps = max(3, min(args.steps, 7))

    def h2d_copy_gbs():
        """The bare host-to-device copy of the batch (pinned), for reference."""
        torch.cuda.synchronize(dev)
        ca, cb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ca.record()
        d_data.copy_(h_data, non_blocking=True)
        cb.record()
        torch.cuda.synchronize(dev)
        return total / (ca.elapsed_time(cb) * 1e-3) / 1e9

    h2d_copy_gbs()
    h2d_before = h2d_copy_gbs()
    d2h = 0
    serial_s = []
    for _ in range(e2e_steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        d_data.copy_(h_data, non_blocking=True)
        d_offs.copy_(h_offs, non_blocking=True)
        step()
        h_co.copy_(d_co, non_blocking=True)
        torch.cuda.synchronize(dev)
        k = int(h_co[-1])
        h_cuts[:k].copy_(d_cuts[:k], non_blocking=True)
        torch.cuda.synchronize(dev)
        serial_s.append(time.perf_counter() - t0)
        d2h = (nfiles + 1) * 8 + k * 8
    e2e_serial_s = statistics.median(serial_s)
    # host check of the last result: CSR is consistent
    assert int(h_co[-1]) == ncuts
    # The host-data entry point: file-aligned pieces with each piece's copy in
    # overlapped with the previous piece's chunking and copy out.
    from paper_2505_21194_gb300.pipeline import HostBatchPipeline, split_files
    pieces = 4
    pipe = HostBatchPipeline(p, tuning, str(dev))
    pipe.run(h_data, offs_np, pieces)
    pipe_s = []
    for _ in range(e2e_steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        hc, hco = pipe.run(h_data, offs_np, pieces)
        pipe_s.append(time.perf_counter() - t0)
    e2e_s = statistics.median(pipe_s)
    e2e_gbs = total * world / e2e_s / 1e9
    assert int(hco[-1]) == ncuts and hc.size == ncuts
    pr = split_files(offs_np.astype(np.int64), pieces)
    d2h_pipe = sum((b - a + 1) * 8 + (int(offs_np[b] - offs_np[a]) // p.min_size + (b - a)) * 8 + 4
                   for a, b in pr)
    # The in-place entry point: the batch stays in pinned host memory and the
    # kernels read it there over the host link (the walk loads only the half
    # windows its scan reaches); the offsets go in, the cut lists come back.
    from paper_2505_21194_gb300.pipeline import HostInPlace
    # (library defaults: the tuning above is the device-resident batch's)
    hip = HostInPlace(p, None, str(dev))
    hip.run(h_data, offs_np)
    inplace_s = []
    for _ in range(e2e_steps):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        hc, hco = hip.run(h_data, offs_np)
        inplace_s.append(time.perf_counter() - t0)
    assert int(hco[-1]) == ncuts and hc.size == ncuts
    ip_stats = seqcdc.seqcdc_stats(hip.ws, walk=seqcdc.seqcdc_algorithm(
        p, total, nfiles, True, hip.ws_bytes, None) == seqcdc.ALGO_WALK)
    ip_path = "chain walk" if "windows" in ip_stats else "segment map"
    # Bytes the kernels read from host memory: the 32-byte sectors the walk
    # loaded, or every byte on the segment map.
    ip_host_bytes = (ip_stats["windows"] * 32 if ip_path == "chain walk" else total)
    inplace_gbs = total * world / statistics.median(inplace_s) / 1e9
    # How busy the host link is: bytes read from host memory per second of
    # the whole call, against the bare host-to-device copy rate.
    ip_link_gbs = ip_host_bytes / statistics.median(inplace_s) / 1e9
    h2d_gbs = h2d_copy_gbs()
    # d_data now holds the batch again (the copies above wrote the same bytes)

    # The same K steps launched directly (one library call per step, its
    # kernels launched one by one), for comparison with the graph.
    direct_ms = None
    if graph is not None:
        for _ in range(3):
            step()
        da, db = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        da.record(stream)
        for _ in range(args.steps):
            step()
        db.record(stream)
        torch.cuda.synchronize(dev)
        direct_ms = da.elapsed_time(db) / args.steps
        if seqcdc.seqcdc_status(d_ws, stream) != 0 or int(d_co[-1].item()) != ncuts:
            direct_ms = None

    # Plain: one seqcdc_chunk call (all kernels) per file, back to back.
    plain_ms = None
    if not args.skip_plain:
        offs64 = offs_np.astype(np.int64)
        cnt = torch.empty(1, dtype=torch.int64, device=dev)
        # one file per call: the library's defaults for a single stream
        ws1 = seqcdc.seqcdc_workspace_size(p, int(np.diff(offs64).max()), 1, None)
        d_ws1 = torch.empty(ws1, dtype=torch.uint8, device=dev)
        # Each file gets its own 16-byte-aligned device buffer (the ABI's
        # alignment rule); file starts inside the CSR batch are arbitrary.
        views = []
        for f in range(nfiles):
            n = int(offs64[f + 1] - offs64[f])
            buf = torch.empty(max(n, 1), dtype=torch.uint8, device=dev)
            buf[:n].copy_(d_data[offs64[f]:offs64[f + 1]])
            views.append(buf[:n])

        def plain_pass():
            for f in range(nfiles):
                seqcdc.seqcdc_chunk(p, views[f], views[f].numel(), d_cuts, cap, cnt,
                                    d_ws1, ws1, None, stream)

        plain_pass()
        torch.cuda.synchronize(dev)
        pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pa.record(stream)
        plain_pass()
        pb.record(stream)
        torch.cuda.synchronize(dev)
        plain_ms = pa.elapsed_time(pb)
        if seqcdc.seqcdc_status(d_ws1, stream) != 0:
            plain_ms = None
        del views
        torch.cuda.empty_cache()
    # The per-file calls wrote into d_cuts: restore this path's output for
    # the fingerprinting below.
    step()
    torch.cuda.synchronize(dev)
    assert int(d_co[-1].item()) == ncuts

    # Fingerprinting the batch's chunks (SHA-256 per chunk) and counting the
    # distinct ones: the step after chunking, on the device.
    fp = None
    if not args.no_fingerprint:
        dig = torch.empty((ncuts, 32), dtype=torch.uint8, device=dev)
        fsz = torch.empty(ncuts, dtype=torch.int32, device=dev)
        fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(2):
            seqcdc.seqcdc_fingerprint_batch(d_data, total, d_offs, nfiles, d_cuts, d_co,
                                            ncuts, dig, fsz, stream)
        reps = 5
        fa.record(stream)
        for _ in range(reps):
            seqcdc.seqcdc_fingerprint_batch(d_data, total, d_offs, nfiles, d_cuts, d_co,
                                            ncuts, dig, fsz, stream)
        fb.record(stream)
        torch.cuda.synchronize(dev)
        fp_ms = fa.elapsed_time(fb) / reps
        nd, nb = seqcdc.dedup(dig, fsz, stream)
        # 1 % of the digests against the host's SHA-256
        import hashlib
        h_cuts = d_cuts[:ncuts].cpu().numpy()
        h_co = d_co.cpu().numpy()
        fidx = np.searchsorted(h_co, np.arange(0, ncuts, 100), side="right") - 1
        hd = dig[::100].cpu().numpy()
        bad = 0
        for j, (i, f) in enumerate(zip(range(0, ncuts, 100), fidx.tolist())):
            a = int(offs_np[f]) + (int(h_cuts[i - 1]) if i > h_co[f] else 0)
            b = int(offs_np[f]) + int(h_cuts[i])
            bad += hd[j].tobytes() != hashlib.sha256(memoryview(data_np)[a:b]).digest()
        fp = {"kernel": "sha256_chunks_kernel", "chunks": ncuts,
              "ms": round(fp_ms, 4), "value": round(total / (fp_ms * 1e-3) / 1e9, 2),
              "unit": "GB/s", "distinct_chunks": nd, "distinct_bytes": nb,
              "checked_vs_host_sha256": len(hd), "mismatches": int(bad)}
        del dig, fsz
    peak, peak_kind = _measured_peaks()
    if walk:
        # The chain walk reads only the scan windows: its algorithmic bytes
        # are the bytes the chain scans (Sec. III.B leaves the rest unread)
        # plus its 4-byte cut records.
        kernel = "walk_kernel"
        span = scan_span_bytes(d_cuts, d_co, ncuts, p)
        alg_bytes = span + ncuts * 4
        # plan_tiles, plan_scan, fill, walk, 3 x (verify, run_repair), verify,
        # repair, count, emit
        launches_per_step = 14
    else:
        kernel = "map_kernel"
        span = None
        alg_bytes = total + ncuts * 8  # each input byte read once + the cut list
        # plan_tiles, plan_scan, map, resolve, 2 x (verify, run_repair), verify,
        # repair, count_tiles, emit
        launches_per_step = 12
    achieved = alg_bytes / (seg_ms * 1e-3) / 1e9
    rec = _traffic_record(kernel)
    traffic = None
    if rec is not None:
        traffic = float(rec["dram_bytes_per_byte"]) * total
    # The other path on the same batch, for comparison (library defaults).
    other = None
    if not args.no_compare:
        alt = seqcdc.Tuning(0, 0, seqcdc.ALGO_MAP if walk else seqcdc.ALGO_WALK, 0)
        ws_alt = seqcdc.seqcdc_workspace_size(p, total, nfiles, alt)
        d_ws_alt = torch.empty(ws_alt, dtype=torch.uint8, device=dev)
        for _ in range(3):
            seqcdc.seqcdc_chunk_batch(p, d_data, total, d_offs, nfiles, d_cuts, cap,
                                      d_co, d_ws_alt, ws_alt, alt, stream)
        oa, ob = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        oa.record(stream)
        for _ in range(reps):
            seqcdc.seqcdc_chunk_batch(p, d_data, total, d_offs, nfiles, d_cuts, cap,
                                      d_co, d_ws_alt, ws_alt, alt, stream)
        ob.record(stream)
        torch.cuda.synchronize(dev)
        o_ms = oa.elapsed_time(ob) / reps
        same = (seqcdc.seqcdc_status(d_ws_alt, stream) == 0 and int(d_co[-1].item()) == ncuts)
        other = {"path": "segment map" if walk else "chain walk", "ms_per_step": round(o_ms, 4),
                 "value": round(total / (o_ms * 1e-3) / 1e9, 2), "unit": "GB/s",
                 "same_cut_count": bool(same)}
        del d_ws_alt
        # restore this path's output for anything below that reads it
        step()
        torch.cuda.synchronize(dev)
    if rank != 0:
        return
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "kernel": kernel,
                "peak_source": peak_kind,
                "kernel_ms": round(seg_ms, 4),
                "algorithmic_bytes": int(alg_bytes),
                "algorithmic": ("scan spans (%d B, %.3f of the input) + 4 B per cut"
                                % (span, span / max(total, 1))) if walk else
                               "every input byte once + 8 B per cut",
                "input_GBs": round(total / (seg_ms * 1e-3) / 1e9, 1),
                "path": "chain walk" if walk else "segment map",
                "piece_bytes": eff.piece_bytes if walk else None,
                "segment_bytes": None if walk else eff.segment_bytes,
                "block_threads": None if walk else eff.block_threads,
                "tuning": tune_src, "cuts": ncuts}
    line = {
        "metric": METRIC,
        "value": round(gbs, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u8",
        "data": "synthetic",
        "config": workload_config(total, nfiles),
        "parallelism": "1 GPU per rank, independent batches (weak scaling)",
        "e2e": {"value": round(inplace_gbs, 2), "unit": "GB/s",
                "h2d_bytes_per_step": int(ip_host_bytes + (nfiles + 1) * 8),
                "d2h_bytes_per_step": int((nfiles + 1) * 8 + ncuts * 8 + 4),
                "api": "pipeline.HostInPlace.run (batch in pinned host memory, read in "
                       "place by the kernels; %s)" % ip_path,
                "input_bytes_on_host": int(total),
                "host_read_GBs": round(ip_link_gbs, 1),
                "host_read_frac_of_copy": round(ip_link_gbs / h2d_before, 3),
                "h2d_bytes": "bytes the kernels read from host memory (32-byte sectors, "
                             "walk counter) + the offsets",
                "copy_pipeline_GBs": round(e2e_gbs, 2),
                "copy_pipeline_api": "pipeline.HostBatchPipeline.run (%d file-aligned pieces, "
                                     "copies overlapped with chunking)" % pieces,
                "copy_pipeline_h2d_bytes_per_step": int(total + (nfiles + 1) * 8),
                "serial_GBs": round(total * world / e2e_serial_s / 1e9, 2),
                "h2d_copy_GBs": round(h2d_before, 1),
                "h2d_copy_GBs_after": round(h2d_gbs, 1),
                "runs": "median of %d" % e2e_steps,
                "host_cpus": ("%d CPUs local to the GPU" % len(numa_cpus)) if numa_cpus
                             else "not bound"},
        "roofline": roofline,
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "launch": ("one CUDA graph of the %d timed steps" % args.steps) if graph is not None
                  else "direct launches",
        "direct_launch_GBs": round(total * world / (direct_ms * 1e-3) / 1e9, 2) if direct_ms else None,
        "plain_loop_GBs": round(total / (plain_ms * 1e-3) / 1e9, 3) if plain_ms else None,
        "batched_vs_plain": round(plain_ms / ms_step, 1) if plain_ms else None,
        "other_path": other["path"] if other else None,
        "other_path_GBs": other["value"] if other else None,
        "fingerprint_GBs": fp["value"] if fp else None,
        "fingerprint_checked": fp["checked_vs_host_sha256"] if fp else None,
        "fingerprint_mismatches": fp["mismatches"] if fp else None,
    }
    detail = {"path_stats": path_stats, "other_path": other, "fingerprint": fp,
              "plain_one_launch_per_file": ({"ms_per_pass": round(plain_ms, 2)}
                                            if plain_ms else None),
              "direct_launch": ({"ms_per_step": round(direct_ms, 4)} if direct_ms else None),
              "e2e_serial_d2h_bytes_per_step": int(d2h)}
    backup = None
    if not args.no_serve or not args.no_dedup or not args.no_single:
        from paper_2505_21194_gb300 import workloads as W
        backup = W.backup_stream(SEED)
    if not args.no_serve:
        # batches of a few ~16 MiB requests: the library's own choice per batch
        sv = serve_levels(dev, p, None, SERVE_LOADS_GBS, backup)
        detail["serve"] = sv
        for lv in sv["levels"]:
            g = lv["offered_GBs"]
            line["serve_%d_p50_ms" % g] = lv["p50_ms"]
            line["serve_%d_p99_ms" % g] = lv["p99_ms"]
            line["serve_%d_sustained_GBs" % g] = lv["sustained_GBs"]
        line["serve_checked"] = sv["checked"]
        line["serve_mismatches"] = sv["mismatches"]
        # Secondary: requests with config 3's log-normal sizes (median
        # 256 KiB), drawn from the 10,000 files already in pinned memory.
        sl = serve_levels(dev, p, None, SERVE_LOGNORMAL_GBS, (data_np, offs_np),
                          pinned=h_data,
                          requests_from="the 10,000 log-normal files of the batch")
        detail["serve_lognormal"] = sl
        for lv in sl["levels"]:
            g = lv["offered_GBs"]
            line["serve_lognormal_%d_p50_ms" % g] = lv["p50_ms"]
            line["serve_lognormal_%d_p99_ms" % g] = lv["p99_ms"]
            line["serve_lognormal_%d_sustained_GBs" % g] = lv["sustained_GBs"]
        line["serve_lognormal_checked"] = sl["checked"]
        line["serve_lognormal_mismatches"] = sl["mismatches"]
    if not args.no_single:
        ss = single_streams(dev, backup, peak, with_cfg5=not args.no_cfg5)
        detail["single_stream"] = ss
        for name, r in ss.items():
            key = name.split("_")[0]
            line["%s_GBs" % key] = r["GBs"]
            line["%s_direct_GBs" % key] = r["direct_GBs"]
            line["%s_path" % key] = r["path"]
            line["%s_kernel_frac" % key] = r["frac"]
            if "host_in_place" in r:
                line["%s_host_in_place_GBs" % key] = r["host_in_place"]["GBs"]
                line["%s_host_in_place_same_cuts" % key] = r["host_in_place"]["same_cuts"]
            if "host_stream" in r:
                line["%s_host_stream_GBs" % key] = r["host_stream"]["GBs"]
                line["%s_host_h2d_copy_GBs" % key] = r["host_stream"]["h2d_copy_GBs"]
                line["%s_host_stream_same_cuts" % key] = r["host_stream"]["same_cuts"]
    if not args.no_dedup:
        dd = dedup_savings(dev, backup)
        sw = sweep_report(dev, backup)
        detail["dedup"], detail["sweep"] = dd, sw
        for r in dd["settings"]:
            suffix = "" if r["mode"] == "increasing" else "_decreasing"
            line["dedup_savings_%dKiB%s" % (r["setting_KiB"], suffix)] = r["savings"]
        line["dedup_host_sha256_agrees"] = all(r["host_sha256_agrees"] for r in dd["settings"])
        sr = sw["search"]
        for reading in (0, 1):
            line["search_table1_mean_KiB_reading%d" % reading] = "/".join(
                "%.2f" % (sr[k]["table1"]["mean_bytes_by_reading"][reading] / 1024)
                for k in (4, 8, 16))
            line["search_settings_within_5pct_reading%d" % reading] = "/".join(
                str(sum(1 for r in sr[k]["within"] if r["reading"] == reading))
                for k in (4, 8, 16))
        for variant in ("seq_length", "seq_length+1", "no_skipping"):
            means = [r["mean_bytes"] / 1024 for r in sw["uniform_random_256MiB"]
                     if r["variant"] == variant]
            line["mean_chunk_KiB_random_%s" % variant.replace("+", "_plus_")] = \
                "/".join("%.2f" % m for m in means)
    if world == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        dt, _ = cpu_oracle_pass(data_np, offs_np, threads)
        reps = 1
        while dt * reps < 10.0 and reps < 4:  # a bounded sample of ~10 s
            d2, _ = cpu_oracle_pass(data_np, offs_np, threads)
            dt += d2
            reps += 1
        # and the single-threaded oracle on a ~1 GB prefix of the batch
        import oracle
        nsamp = int(np.searchsorted(offs_np, 1 << 30))
        t1 = time.perf_counter()
        oracle.chunk_batch(data_np[:int(offs_np[nsamp])], offs_np[:nsamp + 1],
                           oracle.presets(KIB, MODE))
        dt1 = time.perf_counter() - t1
        line["cpu_baseline"] = {
            "value": round(total * reps / dt / 1e9, 3), "unit": "GB/s", "cores": threads,
            "kind": "oracle",
            "sample": "%d pass(es) over the full 10,000-file batch, files spread over "
                      "%d host threads" % (reps, threads),
            "single_thread_GBs": round(int(offs_np[nsamp]) / dt1 / 1e9, 3),
            "single_thread_sample": "the first %d files (%d bytes), one thread"
                                    % (nsamp, int(offs_np[nsamp]))}
    # The verbose detail first (not JSON-parsed), the one JSON line last.
    print("detail: " + json.dumps(detail), flush=True)
    print(json.dumps(line), flush=True)


SERVE_LOADS_GBS = (25, 50, 100, 200)
SERVE_LOGNORMAL_GBS = (10, 25, 50, 100)  # requests of config 3's sizes (many small ones)


def time_stream(dev, d, p, peak, reps=5, flush=None, tuning=None):
    """One device-resident stream chunked by seqcdc_chunk (the library's own
    path choice unless `tuning` says otherwise): median call time and
    dominant-kernel time over `reps` calls (CUDA events on the launching
    stream; `flush`, a tensor larger than L2, is rewritten before each call),
    the path, the cut count and the dominant kernel's roofline fraction."""
    import torch
    from paper_2505_21194_gb300 import seqcdc
    n = d.numel()
    cap = n // p.min_size + 1
    cuts = torch.empty(max(cap, 1), dtype=torch.int64, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ws_bytes = seqcdc.seqcdc_workspace_size(p, n, 1, tuning)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    algo = seqcdc.seqcdc_algorithm(p, n, 1, False, ws_bytes, tuning)

    def call(st=None):
        seqcdc.seqcdc_chunk(p, d, n, cuts, cap, cnt, ws, ws_bytes, tuning, st or stream)

    for _ in range(3):
        call()
    if seqcdc.seqcdc_status(ws, stream) != 0:
        raise RuntimeError("device status during warm-up")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in ev:
        e.record(stream)
    # The call captured once in a CUDA graph (its kernels launched as one
    # graph, the dominant kernel bracketed by events on every replay).
    gs = torch.cuda.Stream(dev)
    gs.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gs):
        call(gs)
        gs.synchronize()
        with torch.cuda.graph(graph, stream=gs):
            seqcdc.seqcdc_profile_events(ev[2], ev[3])
            call(gs)
        seqcdc.seqcdc_profile_events(None, None)
    stream.wait_stream(gs)

    def timed(use_graph):
        steps, kern = [], []
        for _ in range(reps):
            if flush is not None:
                flush.add_(1)
            ev[0].record(stream)
            if use_graph:
                graph.replay()
            else:
                seqcdc.seqcdc_profile_events(ev[2], ev[3])
                call()
                seqcdc.seqcdc_profile_events(None, None)
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            steps.append(ev[0].elapsed_time(ev[1]))
            kern.append(ev[2].elapsed_time(ev[3]))
        return steps, kern

    dsteps, _ = timed(False)
    steps, kern = timed(True)
    if seqcdc.seqcdc_status(ws, stream) != 0:
        raise RuntimeError("device status in the timed calls")
    del graph
    k = int(cnt.item())
    ms, kms = statistics.median(steps), statistics.median(kern)
    walk = algo == seqcdc.ALGO_WALK
    if walk:
        co = torch.tensor([0, k], dtype=torch.int64, device=dev)
        alg = scan_span_bytes(cuts, co, k, p) + 4 * k
    else:
        alg = n + 8 * k
    del ws, cuts
    dms = statistics.median(dsteps)
    return {"GBs": round(n / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 4),
            "launch": "CUDA graph of one call",
            "direct_GBs": round(n / (dms * 1e-3) / 1e9, 2), "direct_ms": round(dms, 4),
            "path": "chain walk" if walk else "segment map",
            "kernel": "walk_kernel" if walk else "map_kernel",
            "kernel_ms": round(kms, 4), "cuts": k, "bytes": n,
            "frac": round(alg / (kms * 1e-3) / 1e9 / peak, 4),
            "algorithmic_bytes": int(alg)}


def single_streams(dev, backup, peak, with_cfg5=True):
    """The single-stream workloads: 16 MiB of uniform random bytes (seed 0,
    8 KiB setting; L2 flushed before every call), the ~1 GiB backup-like
    stream (8 KiB setting, increasing) and the 64 GiB adversarial stream
    (16 KiB setting), each in one seqcdc_chunk call."""
    import torch
    from paper_2505_21194_gb300 import seqcdc, workloads as W
    out = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    d = torch.from_numpy(W.uniform_random(16 << 20, SEED)).to(dev)
    out["cfg1_16MiB_random"] = time_stream(dev, d, seqcdc.seqcdc_params(8, 0), peak,
                                           reps=7, flush=flush)
    del d, flush
    d = torch.from_numpy(backup[0]).to(dev)
    out["cfg2_1GiB_backup"] = time_stream(dev, d, seqcdc.seqcdc_params(8, 0), peak)
    # The same stream fed from pinned host memory in 128 MiB blocks through the
    # resumable stream pipeline (copies overlapped with chunking), against the
    # bare host-to-device copy of the same bytes.
    from paper_2505_21194_gb300.pipeline import HostStreamPipeline
    h = torch.from_numpy(backup[0]).pin_memory()
    n = h.numel()
    pipe = HostStreamPipeline(seqcdc.seqcdc_params(8, 0), device=str(dev))
    blocks = [h[a:a + (128 << 20)] for a in range(0, n, 128 << 20)]
    ref = pipe.run(blocks)
    ts, tc = [], []
    for _ in range(3):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        got = pipe.run(blocks)
        ts.append(time.perf_counter() - t)
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        d.copy_(h, non_blocking=True)
        torch.cuda.synchronize(dev)
        tc.append(time.perf_counter() - t)
    same = bool(got.size == out["cfg2_1GiB_backup"]["cuts"] and np.array_equal(got, ref))
    out["cfg2_1GiB_backup"]["host_stream"] = {
        "GBs": round(n / statistics.median(ts) / 1e9, 2),
        "h2d_copy_GBs": round(n / statistics.median(tc) / 1e9, 2),
        "same_cuts": same, "blocks": len(blocks),
        "api": "pipeline.HostStreamPipeline.run, 128 MiB pinned blocks, median of 3"}
    # The same pinned stream read in place by the kernels (no copy of it).
    from paper_2505_21194_gb300.pipeline import HostInPlace
    hip = HostInPlace(seqcdc.seqcdc_params(8, 0), device=str(dev))
    hip.run_stream(h)
    ti = []
    for _ in range(3):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        got_ip = hip.run_stream(h)
        ti.append(time.perf_counter() - t)
    out["cfg2_1GiB_backup"]["host_in_place"] = {
        "GBs": round(n / statistics.median(ti) / 1e9, 2),
        "same_cuts": bool(np.array_equal(got_ip, ref)),
        "api": "pipeline.HostInPlace.run_stream, median of 3"}
    del d, h, pipe, hip
    if with_cfg5:
        block, nblocks = 16 << 20, 4096
        d = torch.empty(block * nblocks, dtype=torch.uint8, device=dev)
        for i in range(nblocks):
            d[i * block:(i + 1) * block].copy_(
                torch.from_numpy(W.adversarial_block(i, SEED, block)))
        out["cfg5_64GiB_adversarial"] = time_stream(dev, d, seqcdc.seqcdc_params(16, 0),
                                                    peak, reps=3)
        del d
    torch.cuda.empty_cache()
    return out


def sweep_report(dev, backup):
    """Mean chunk size at Table I's settings on uniform random bytes and on
    the backup-like stream: as read here (a run of SeqLength bytes), with one
    more byte per run (the other reading), and without skipping (BASE)."""
    import torch
    from paper_2505_21194_gb300 import workloads as W
    from paper_2505_21194_gb300.sweep import sweep, table1_settings
    out = {}
    samples = (("uniform_random_256MiB", W.uniform_random(256 << 20, SEED + 7)),
               ("backup_stream_1GiB", backup[0]))
    for name, arr in samples:
        d = torch.from_numpy(arr).to(dev)
        rows = []
        for label, sets in (("seq_length", table1_settings()),
                            ("seq_length+1", table1_settings(extra_run_byte=True)),
                            ("no_skipping", table1_settings(base=True))):
            for kib, r in zip((4, 8, 16), sweep(d, sets)):
                rows.append({"setting_KiB": kib, "variant": label,
                             "mean_bytes": r["mean_bytes"], "at_max": r["at_max"]})
        out[name] = rows
        del d
    # Sec. V's Monte-Carlo search: SeqLength 3..8 x SkipTrigger 20..80 (step
    # 5) x SkipSize 128/256/512, Sec. VI's min / max, both readings of
    # SeqLength, on 64 MiB of uniform random bytes.
    from paper_2505_21194_gb300.sweep import search
    d = torch.from_numpy(W.uniform_random(64 << 20, SEED + 9)).to(dev)
    t = time.perf_counter()
    out["search"] = search(d)
    out["search_s"] = round(time.perf_counter() - t, 2)
    del d
    return out


def dedup_savings(dev, backup):
    """Deduplication savings of the ~1 GiB backup-like stream (64 edited
    versions of a 16 MiB base) chunked, fingerprinted (SHA-256) and counted
    on the GPU at the three settings in both modes: 1 - (bytes of distinct
    chunks) / (all bytes) (Eq. 1); the host's SHA-256 recounts the same
    chunks as the check."""
    import hashlib
    from concurrent.futures import ThreadPoolExecutor
    import torch
    from paper_2505_21194_gb300 import seqcdc
    stream, _ = backup
    d = torch.from_numpy(stream).to(dev)
    o = torch.tensor([0, stream.size], dtype=torch.int64, device=dev)
    mv = memoryview(stream)
    out = []
    with ThreadPoolExecutor(os.cpu_count() or 1) as pool:
        for kib in (4, 8, 16):
            for mode in (0, 1):
                p = seqcdc.seqcdc_params(kib, mode)
                r = seqcdc.chunk_batch(d, o, p)
                dig, sz = seqcdc.fingerprint(d, o, r)
                gpu_chunks, gpu_bytes = seqcdc.dedup(dig, sz)
                cuts = r.cuts.cpu().numpy()
                del dig, sz, r
                starts = np.concatenate([[0], cuts[:-1]])
                digests = list(pool.map(
                    lambda ab: hashlib.sha256(mv[ab[0]:ab[1]]).digest(),
                    zip(starts.tolist(), cuts.tolist()), chunksize=256))
                seen, unique = set(), 0
                for (a, b), h in zip(zip(starts.tolist(), cuts.tolist()), digests):
                    if h not in seen:
                        seen.add(h)
                        unique += b - a
                out.append({"setting_KiB": kib, "mode": "increasing" if mode == 0 else "decreasing",
                            "chunks": int(cuts.size),
                            "mean_chunk_B": round(stream.size / max(cuts.size, 1), 1),
                            "savings": round(1.0 - gpu_bytes / stream.size, 4),
                            "distinct_chunks": gpu_chunks,
                            "host_sha256_agrees": bool(gpu_bytes == unique and
                                                       gpu_chunks == len(seen))})
    del d
    return {"stream": "64 versions of a 16 MiB base, Poisson(200) edits each "
                      "(%d bytes)" % stream.size,
            "hash": "SHA-256 per chunk and distinct-chunk table on the GPU; "
                    "host SHA-256 (hashlib) as the check", "settings": out}


def serve_levels(dev, p, tuning, loads, backup, duration_s=1.0, pinned=None,
                 requests_from="64 versions (~16 MiB each) of the 1 GiB backup-like stream",
                 reps=3):
    """Open-loop serving at each offered load (GB/s): Poisson arrivals of
    requests drawn from the payloads of ``backup`` (bytes, offsets: by
    default the 64 versions, about 16 MiB each, of the backup-like stream;
    ``pinned`` may hold the same bytes already in pinned memory), admitted
    under a 64 GiB HBM budget, batched continuously.  One request in a
    hundred is checked against the oracle and against the same payload
    chunked alone."""
    import torch
    import oracle
    from paper_2505_21194_gb300 import seqcdc, workloads as W
    from paper_2505_21194_gb300.serve import Server, poisson_arrivals
    stream, voffs = backup
    voffs = voffs.astype(np.int64)
    sizes = np.diff(voffs)
    pool = pinned if pinned is not None else torch.from_numpy(stream).pin_memory()
    srv = Server(p, pool, voffs, budget_bytes=64 << 30, max_batch_bytes=4 << 30,
                 tuning=tuning, device=str(dev))
    op = oracle.Params(p.mode, p.seq_length, p.skip_trigger, p.skip_size,
                       p.min_size, p.max_size)
    expect, alone = {}, {}
    levels, checked, bad = [], 0, 0
    srv.run(poisson_arrivals(20.0, 0.2, len(sizes), sizes, SEED))  # warm-up
    for gbs in loads:
        rate = gbs * 1e9 / float(sizes.mean())
        arr = poisson_arrivals(rate, duration_s, len(sizes), sizes, SEED + int(gbs))
        keep = {r.rid for r in arr if r.rid % 100 == 0}
        # The same arrivals served `reps` times: the medians are reported,
        # every run's p99 is kept (a 1 s window's p99 moves with anything
        # else the shared host does meanwhile).
        runs = []
        for _ in range(reps):
            st = srv.run(arr, keep=keep)
            runs.append(st)
            for r in arr:
                if r.rid not in keep:
                    continue
                k = r.payload
                if k not in expect:
                    b = stream[voffs[k]:voffs[k + 1]]
                    expect[k] = oracle.chunk(b, op).astype(np.int64)
                    alone[k] = seqcdc.chunk(torch.from_numpy(b).to(dev), p, tuning).cpu().numpy()
                got = st.results[r.rid].cpu().numpy()
                checked += 1
                bad += int(not (np.array_equal(got, expect[k]) and np.array_equal(got, alone[k])))
        med = lambda xs: float(np.median(xs))
        levels.append({"offered_GBs": gbs, "requests": runs[0].requests,
                       "batches": [st.batches for st in runs],
                       "sustained_GBs": round(med([st.sustained_gbs for st in runs]), 2),
                       "p50_ms": round(med([st.latency["p50_ms"] for st in runs]), 3),
                       "p99_ms": round(med([st.latency["p99_ms"] for st in runs]), 3),
                       "p99_ms_each_run": [round(st.latency["p99_ms"], 3) for st in runs]})
    return {"requests_from": requests_from,
            "arrivals": "Poisson, open loop, %.1f s per level, %d runs of each level "
                        "(medians reported)" % (duration_s, reps),
            "hbm_budget_GiB": 64, "max_batch_GiB": 4, "levels": levels,
            "checked": checked, "mismatches": bad,
            "latency": "arrival to completion of the batch's chunking (device clock); "
                       "cut lists stay on the device"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--segment-bytes", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--algorithm", default="auto", choices=["auto", "map", "walk"],
                    help="chunking path (default: autotuned, else the library's AUTO rule)")
    ap.add_argument("--piece-bytes", type=int, default=0,
                    help="chain walk: bytes per piece (0 = library default)")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the other chunking path on the same batch")
    ap.add_argument("--no-cpu", action="store_true",
                    help="skip the CPU-oracle baseline (profiling runs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="library default launch tuning instead of the autotuner")
    ap.add_argument("--no-fingerprint", action="store_true",
                    help="skip SHA-256 fingerprinting of the batch's chunks")
    ap.add_argument("--no-dedup", action="store_true",
                    help="skip the deduplication-savings report on the backup-like stream")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving measurement (open-loop Poisson arrivals)")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the timed steps directly instead of as one CUDA graph")
    ap.add_argument("--no-single", action="store_true",
                    help="skip the single-stream workloads (16 MiB, 1 GiB, 64 GiB)")
    ap.add_argument("--no-cfg5", action="store_true",
                    help="skip the 64 GiB adversarial stream among the single streams")
    ap.add_argument("--nfiles", type=int, default=NFILES,
                    help="files in the batch (default: the 10,000-file workload)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
