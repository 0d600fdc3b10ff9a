"""One stream chunked by several ranks: contiguous ranges, one exchange of
each range's exit, junction walks at the range starts, rounds until no exit
changes.  On the CPU the ranks are gloo processes and the oracle is their
chunker; on the GPU the library's kernels chunk the ranges."""
from __future__ import annotations

import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_2505_21194_gb300 import multistream as ms
from paper_2505_21194_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KIB, MIB = 1 << 10, 1 << 20


def _stream(case: int) -> np.ndarray:
    """Random and text-like stretches with a long constant run and a ramp:
    a range inside the constant run never meets its own spec walk."""
    rng = np.random.default_rng(case)
    parts = [rng.integers(0, 256, 600 * KIB, dtype=np.uint8),
             np.zeros(2 * MIB + 123, dtype=np.uint8),
             W.mixed_base(700 * KIB, case),
             np.tile(np.arange(256, dtype=np.uint8), 2048),
             rng.integers(0, 256, 900 * KIB + 77, dtype=np.uint8)]
    return np.concatenate(parts)


def _oracle_fn(op):
    return lambda b: oracle.chunk(np.ascontiguousarray(b), op).astype(np.int64)


def test_split_ranges_contiguous_and_aligned():
    for n, world, align in ((10 * MIB + 5, 3, MIB), (1000, 4, 64), (5, 3, 16), (0, 2, 16)):
        r = ms.split_ranges(n, world, align)
        assert len(r) == world and r[0][0] == 0 and r[-1][1] == n
        assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))
        assert all(a % align == 0 for a, _ in r)
        assert all(b >= a for a, b in r)


@pytest.mark.parametrize("mode", [0, 1])
def test_ranges_one_process_equal_the_oracle(mode):
    """Every split of the stream gives the oracle's cut list of the whole
    stream; a range inside the constant run takes a second round."""
    op = oracle.presets(8, mode)
    data = _stream(3)
    n = data.size
    want = oracle.chunk(data, op).astype(np.int64)
    fn = _oracle_fn(op)
    for world, align in ((1, 4096), (2, 4096), (3, 4096), (5, 64 * KIB), (7, 16)):
        ranges = ms.split_ranges(n, world, align)
        bufs = [data[slice(*ms.held_bytes(a, b, n, op))] for a, b in ranges]
        got, _ = ms.chunk_stream_ranges(bufs, ranges, n, op, fn)
        assert np.array_equal(got, want), (world, align)
    # ranges boundaries inside the zero run: its ranges' exits change
    ranges = [(0, 700 * KIB), (700 * KIB, 1600 * KIB), (1600 * KIB, 2400 * KIB), (2400 * KIB, n)]
    bufs = [data[slice(*ms.held_bytes(a, b, n, op))] for a, b in ranges]
    got, rounds = ms.chunk_stream_ranges(bufs, ranges, n, op, fn)
    assert np.array_equal(got, want)
    assert rounds >= 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2505_21194_gb300 import multistream as m
    import oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        op = orc.presets(8, 0)
        data = _stream(3)
        n = data.size
        ranges = m.split_ranges(n, world, 4096) if world != 4 else [
            (0, 700 * KIB), (700 * KIB, 1600 * KIB), (1600 * KIB, 2400 * KIB), (2400 * KIB, n)]
        a, b = ranges[rank]
        buf = data[slice(*m.held_bytes(a, b, n, op))]
        got = m.chunk_stream_distributed(buf, a, b, n, op, _oracle_fn(op), device="cpu")
        q.put((rank, got.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_ranges_gloo_ranks_equal_the_oracle(world):
    """Real ranks (gloo, one process each): the exchange of exits and the
    rounds give the oracle's cut list; world 4 puts a range inside the zero
    run, so its exit changes and the next rank walks again."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = dict(q.get(timeout=300) for _ in range(world))
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    got = np.concatenate([np.asarray(res[r], dtype=np.int64) for r in range(world)])
    want = oracle.chunk(_stream(3), oracle.presets(8, 0)).astype(np.int64)
    assert np.array_equal(got, want)


@pytest.mark.gpu
def test_ranges_on_the_library_equal_one_call(gpu):
    """The ranges chunked by the library's kernels (junction walks from
    unaligned cuts included) give the cut list of one call on the whole
    stream, in both modes."""
    import torch
    s = gpu
    data = _stream(3)
    n = data.size
    d = torch.from_numpy(data).cuda()
    zero_split = [(0, 700 * KIB), (700 * KIB, 1600 * KIB), (1600 * KIB, 2400 * KIB),
                  (2400 * KIB, n)]
    for mode in (0, 1):
        p = s.seqcdc_params(8, mode)
        want = s.chunk(d, p).cpu().numpy()
        for ranges in (ms.split_ranges(n, 3, 4096), zero_split):
            bufs = [d[slice(*ms.held_bytes(a, b, n, p))] for a, b in ranges]
            got, _ = ms.chunk_stream_ranges(bufs, ranges, n, p)
            assert np.array_equal(got, want), (mode, ranges)


def test_ranges_shorter_than_max_size_equal_the_oracle():
    """Ranges of a few KiB, below max_size: one chunk spans several ranges,
    so a range is entered at or past its own end and passes that cut on."""
    op = oracle.presets(8, 0)
    rng = np.random.default_rng(9)
    data = np.concatenate([rng.integers(0, 256, 150 * KIB, dtype=np.uint8),
                           np.zeros(60 * KIB, dtype=np.uint8),
                           rng.integers(0, 256, 50 * KIB + 3, dtype=np.uint8)])
    n = data.size
    want = oracle.chunk(data, op).astype(np.int64)
    for world, align in ((20, 16), (37, 64), (64, 16)):
        ranges = ms.split_ranges(n, world, align)
        assert max(b - a for a, b in ranges) < op.max_size
        bufs = [data[slice(*ms.held_bytes(a, b, n, op))] for a, b in ranges]
        got, _ = ms.chunk_stream_ranges(bufs, ranges, n, op, _oracle_fn(op))
        assert np.array_equal(got, want), world


def _failing_rank_main(rank, world, port, q, how):
    """Rank 1 fails between init and the exchange (``exit``: the process
    ends; ``stall``: it never joins); rank 0 runs the exchange under a
    5-second process-group timeout and reports what it got."""
    import datetime
    import time
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2505_21194_gb300 import multistream as m
    import oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        if how == "exit":
            os._exit(3)
        time.sleep(15)
        os._exit(4)
    op = orc.presets(8, 0)
    data = _stream(3)
    n = data.size
    a, b = m.split_ranges(n, world, 4096)[0]
    buf = data[slice(*m.held_bytes(a, b, n, op))]
    t0 = time.monotonic()
    try:
        m.chunk_stream_distributed(buf, a, b, n, op, _oracle_fn(op), device="cpu")
        q.put(("returned", "", time.monotonic() - t0))
    except Exception as e:  # the failure must surface as an exception
        q.put(("raised", type(e).__name__, time.monotonic() - t0))
    q.close()
    q.join_thread()
    os._exit(0)


@pytest.mark.parametrize("how", ["exit", "stall"])
def test_a_failed_rank_ends_the_exchange_with_an_error(how):
    """A rank that exits, or stalls, before the exchange of exits: the other
    rank's exchange ends with an exception within the process group's
    timeout instead of waiting forever, and no cut list is returned."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_failing_rank_main, args=(r, 2, port, q, how))
             for r in range(2)]
    for pr in procs:
        pr.start()
    try:
        kind, name, secs = q.get(timeout=150)
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.kill()
                pr.join()
    assert kind == "raised", (kind, name)
    assert secs < 60, secs
    assert procs[0].exitcode == 0
