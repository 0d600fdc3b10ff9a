"""Host-resident data: pipelined batches and resumable streams."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle
from paper_2505_21194_gb300 import workloads as W
from paper_2505_21194_gb300.pipeline import split_files


def _check_split(offs, pieces):
    r = split_files(np.asarray(offs), pieces)
    nf = len(offs) - 1
    assert r[0][0] == 0 and r[-1][1] == nf
    assert all(b > a for a, b in r)
    assert all(r[k][1] == r[k + 1][0] for k in range(len(r) - 1))
    assert len(r) <= max(1, min(pieces, nf))
    return r


def test_split_files_balanced_and_whole():
    offs = np.concatenate([[0], np.cumsum(np.full(100, 10))])
    r = _check_split(offs, 4)
    assert [b - a for a, b in r] == [25, 25, 25, 25]
    _check_split(offs, 1)
    _check_split(offs, 100)
    _check_split(offs, 500)                       # more pieces than files
    big = np.array([0, 1000, 1001, 1002, 1003])   # one large file first
    r = _check_split(big, 3)
    assert r[0] == (0, 1)
    assert split_files(np.array([0]), 4) == []
    _check_split(np.array([0, 0, 0, 5]), 2)       # empty files


@pytest.mark.gpu
def test_chunk_batch_host_equals_device_batch(gpu):
    import torch
    from paper_2505_21194_gb300.pipeline import chunk_batch_host
    s = gpu
    data, offs = W.file_batch(40, seed=8)
    offs = offs.astype(np.int64)
    offs = np.insert(offs, 5, offs[5])            # an empty file
    p = s.seqcdc_params(8, 0)
    r = s.chunk_batch(torch.from_numpy(data).cuda(), torch.from_numpy(offs).cuda(), p)
    exp_c, exp_co = r.cuts.cpu().numpy(), r.cut_offsets.cpu().numpy()
    h = torch.from_numpy(data).pin_memory()
    for pieces in (1, 3, 7, 64):
        c, co = chunk_batch_host(h, offs, p, pieces=pieces)
        assert np.array_equal(co, exp_co) and np.array_equal(c, exp_c), pieces
    ec, eco = oracle.chunk_batch(data, offs.astype(np.uint64), oracle.presets(8))
    assert np.array_equal(exp_c, ec.astype(np.int64))


@pytest.mark.gpu
def test_chunk_stream_host_equals_oracle(gpu):
    from paper_2505_21194_gb300.pipeline import chunk_stream_host
    s = gpu
    rng = np.random.default_rng(4)
    data = W.mixed_base(12 << 20, 9)
    data[3 << 20:(3 << 20) + 200000] = 0          # a stretch without runs
    sizes = rng.integers(1, 3 << 20, 20)
    cutsz = np.minimum(np.cumsum(sizes), data.size)
    blocks = np.split(data, np.unique(cutsz[:-1]))
    for kib in (4, 16):
        p = s.seqcdc_params(kib, 1)
        got = np.concatenate(list(chunk_stream_host(iter(blocks), p)))
        exp = oracle.chunk(data, oracle.presets(kib, 1)).astype(np.int64)
        assert np.array_equal(got, exp)


@pytest.mark.gpu
def test_host_pipeline_reused_and_growing(gpu):
    import torch
    from paper_2505_21194_gb300.pipeline import HostBatchPipeline
    s = gpu
    p = s.seqcdc_params(4, 0)
    pipe = HostBatchPipeline(p, slots=2)
    for nf, seed in ((12, 1), (60, 2), (5, 3)):          # the second batch is larger
        data, offs = W.file_batch(nf, seed=seed)
        offs = offs.astype(np.int64)
        r = s.chunk_batch(torch.from_numpy(data).cuda(), torch.from_numpy(offs).cuda(), p)
        c, co = pipe.run(torch.from_numpy(data).pin_memory(), offs, pieces=4)
        assert np.array_equal(co, r.cut_offsets.cpu().numpy())
        assert np.array_equal(c, r.cuts.cpu().numpy())


@pytest.mark.gpu
def test_host_stream_pipeline_resumable_uneven_blocks(gpu):
    """A 40 MiB stream through 4 MiB slots in uneven blocks (one larger than
    a slot, some of a few bytes), with a stretch of constant bytes (no run
    ends: every cut there is forced at max_size): after every feed the cuts
    returned so far are a prefix of the oracle's; the whole list equals it;
    the pipeline is reused for a second stream (numpy blocks this time)."""
    import torch
    from paper_2505_21194_gb300.pipeline import HostStreamPipeline
    s = gpu
    rng = np.random.default_rng(11)
    data = W.mixed_base(40 << 20, 12)
    data[(9 << 20):(9 << 20) + 700000] = 7
    for kib, mode in ((8, 0), (16, 1)):
        p = s.seqcdc_params(kib, mode)
        exp = oracle.chunk(data, oracle.presets(kib, mode)).astype(np.int64)
        pipe = HostStreamPipeline(p, block_bytes=4 << 20)
        h = torch.from_numpy(data).pin_memory()
        bounds = [0, 3, 17, 5 << 20, (5 << 20) + 1, 11 << 20, 19 << 20, 19 << 20,
                  (30 << 20) + 12345, data.size]
        got = []
        for a, b in zip(bounds[:-1], bounds[1:]):
            got.append(pipe.feed(h[a:b]))
            so_far = np.concatenate(got)
            assert np.array_equal(so_far, exp[:so_far.size])
            assert so_far.size == 0 or so_far[-1] <= b
        got.append(pipe.finish())
        assert np.array_equal(np.concatenate(got), exp)
        # reuse: the same stream again, in numpy blocks of random sizes
        cut = np.unique(rng.integers(0, data.size, 7))
        blocks = np.split(data, cut)
        assert np.array_equal(pipe.run(blocks), exp)


@pytest.mark.gpu
def test_host_in_place_equals_device_and_oracle(gpu):
    """Input read in place from pinned host memory: the same cuts as on the
    device, on both paths (AUTO takes the walk for host input), for a batch
    with an empty file and a stream; pageable input is refused."""
    import torch
    from paper_2505_21194_gb300.pipeline import HostInPlace
    s = gpu
    data, offs = W.file_batch(300, seed=21)
    offs = np.insert(offs.astype(np.int64), 7, offs[7])   # an empty file
    p = s.seqcdc_params(8, 0)
    r = s.chunk_batch(torch.from_numpy(data).cuda(), torch.from_numpy(offs).cuda(), p)
    exp_c, exp_co = r.cuts.cpu().numpy(), r.cut_offsets.cpu().numpy()
    h = torch.from_numpy(data).pin_memory()
    hp = HostInPlace(p)
    for tuning in (None, s.Tuning(0, 0, s.ALGO_WALK, 262144), s.Tuning(0, 0, s.ALGO_MAP, 0)):
        hp.tuning = tuning
        hp.max_bytes = -1                                 # workspace for this tuning
        c, co = hp.run(h, offs)
        assert np.array_equal(co, exp_co) and np.array_equal(c, exp_c), tuning
    # convenience entry points take the pinned tensor as it is
    r2 = s.chunk_batch(h, torch.from_numpy(offs), p)
    assert torch.equal(r2.cuts.cpu(), r.cuts.cpu())
    a, b = int(offs[2]), int(offs[3])
    ec = oracle.chunk(data[a:b], oracle.presets(8)).astype(np.int64)
    assert np.array_equal(exp_c[exp_co[2]:exp_co[3]], ec)
    # one stream, both modes
    stream = W.mixed_base(24 << 20, 5)
    hs = torch.from_numpy(stream).pin_memory()
    for mode in (0, 1):
        q = s.seqcdc_params(8, mode)
        hq = HostInPlace(q)
        got = hq.run_stream(hs)
        want = s.chunk(torch.from_numpy(stream).cuda(), q).cpu().numpy()
        assert np.array_equal(got, want), mode
        assert np.array_equal(s.chunk(hs, q).cpu().numpy(), want)
    # pageable host memory cannot be read by the device: refused, not launched
    with pytest.raises(TypeError):
        s.chunk(torch.from_numpy(stream), p)
    lib = s.load_library()
    pageable = torch.from_numpy(stream.copy())
    n = pageable.numel()
    ws_bytes = s.seqcdc_workspace_size(p, n, 1)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    cuts = torch.empty(n // p.min_size + 1, dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = lib.seqcdc_chunk(ctypes.byref(p), pageable.data_ptr(), n, cuts.data_ptr(),
                          cuts.numel(), cnt.data_ptr(), ws.data_ptr(), ws_bytes, None, None)
    assert rc == s.SEQCDC_EINVAL


@pytest.mark.gpu
def test_host_in_place_tiny_and_ragged_streams(gpu):
    """Streams read in place whose sizes are empty, below a 16-byte load,
    not a multiple of 16, and around min_size and max_size: the same cuts
    as on the device, and the oracle's."""
    import torch
    from paper_2505_21194_gb300.pipeline import HostInPlace
    s = gpu
    p = s.seqcdc_params(8, 0)
    hp = HostInPlace(p)
    base = W.mixed_base(1 << 20, 11)
    for n in (0, 1, 15, 17, 4095, 4096, 4097, 16383, 16384, 16385, 70001, (1 << 20) - 3):
        data = base[:n].copy()
        h = torch.from_numpy(data).pin_memory() if n else torch.empty(0, dtype=torch.uint8)
        got = hp.run_stream(h)
        want = oracle.chunk(data, oracle.presets(8)).astype(np.int64) if n else np.zeros(0, np.int64)
        assert np.array_equal(got, want), n
        if n:
            dev = s.chunk(torch.from_numpy(data).cuda(), p).cpu().numpy()
            assert np.array_equal(dev, want), n


@pytest.mark.gpu
def test_host_in_place_other_seq_lengths_and_no_skipping(gpu):
    """The host chunk step's general SeqLength path (not 5) and the path
    without skipping (SkipTrigger 0): the same cuts as on the device and the
    oracle's, in both modes."""
    import torch
    from paper_2505_21194_gb300.pipeline import HostInPlace
    s = gpu
    data = W.mixed_base(6 << 20, 13)
    h = torch.from_numpy(data).pin_memory()
    d = torch.from_numpy(data).cuda()
    for mode in (0, 1):
        for R, T, S in ((3, 40, 128), (8, 30, 256), (16, 0, 0), (5, 0, 0)):
            p = s.Params(mode, R, T, S, 4096, 16384)
            op = oracle.Params(mode, R, T, S, 4096, 16384)
            want = oracle.chunk(data, op).astype(np.int64)
            got = HostInPlace(p).run_stream(h)
            assert np.array_equal(got, want), (mode, R, T, S)
            walk = (0, 0, s.ALGO_WALK, 262144)
            assert np.array_equal(s.chunk(d, p, walk).cpu().numpy(), want), (mode, R, T, S)
