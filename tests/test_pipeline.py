"""Host-resident data: pipelined batches and resumable streams."""
from __future__ import annotations

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
