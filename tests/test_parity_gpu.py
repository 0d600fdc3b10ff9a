"""GPU parity: the CUDA chunker against the CPU oracle, element by element.

Inputs are seeded and synthetic.  Small cases force many segments (4 KiB
segments) so junctions, look-back and replay all run; full-size cases use the
benchmark workloads and their launch configuration."""
from __future__ import annotations

import json
import os

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2505_21194_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _p(s, p: Params):
    return s.make_params(p.mode, p.seq_length, p.skip_trigger, p.skip_size,
                         p.min_size, p.max_size)


def gpu_chunk(s, b: np.ndarray, p: Params, seg=0, threads=0):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    cuts = s.chunk(d, _p(s, p), tuning=(seg, threads))
    return cuts.cpu().numpy().astype(np.uint64)


def gpu_batch(s, data, offs, p: Params, seg=0, threads=0):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    o = torch.from_numpy(np.asarray(offs, dtype=np.int64)).cuda()
    r = s.chunk_batch(d, o, _p(s, p), tuning=(seg, threads))
    return r.cuts.cpu().numpy().astype(np.uint64), r.cut_offsets.cpu().numpy().astype(np.uint64)


def assert_same(got, exp):
    got = np.asarray(got, dtype=np.uint64)
    exp = np.asarray(exp, dtype=np.uint64)
    if got.size != exp.size or not np.array_equal(got, exp):
        k = int(np.argmax(got[:min(got.size, exp.size)] != exp[:min(got.size, exp.size)])) \
            if min(got.size, exp.size) else 0
        raise AssertionError("cut lists differ: %d vs %d cuts, first difference at "
                             "index %d: gpu %s oracle %s" % (
                                 got.size, exp.size, k, got[k:k + 4].tolist(),
                                 exp[k:k + 4].tolist()))


@pytest.mark.parametrize("name", ["hand_example.json", "trigger_example.json",
                                  "vector_example.json"])
def test_worked_examples(gpu, name):
    with open(os.path.join(GOLDEN, name)) as f:
        d = json.load(f)
    p = Params(**d["params"])
    b = np.array(d["bytes"], np.uint8)
    assert gpu_chunk(gpu, b, p, seg=4096).tolist() == d["cuts"]


@pytest.mark.parametrize("seed", range(40))
def test_random_small_many_segments(gpu, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 200000))
    kind = seed % 4
    if kind == 0:
        b = rng.integers(0, 256, n).astype(np.uint8)
    elif kind == 1:
        b = rng.integers(0, 3, n).astype(np.uint8)
    elif kind == 2:
        b = W.markov_text(n, seed)
    else:
        b = W.mixed_base(n, seed, block=8192) if n else np.empty(0, np.uint8)
    R = int(rng.integers(2, 8))
    mn = int(rng.integers(1, 3000))
    mx = int(rng.integers(mn, min(mn + 9000, 65536)))
    p = Params(int(rng.integers(0, 2)), R, int(rng.integers(0, 60)),
               int(rng.integers(0, 600)), mn, mx)
    seg = int(rng.choice([4096, 8192, 16384]))
    assert_same(gpu_chunk(gpu, b, p, seg=seg), oracle.chunk(b, p))


@pytest.mark.parametrize("kib", [4, 8, 16])
@pytest.mark.parametrize("mode", [0, 1])
def test_presets_edge_lengths(gpu, kib, mode):
    p = oracle.presets(kib, mode)
    rng = np.random.default_rng(kib * 10 + mode)
    L = 65536
    for n in (0, 1, 2, p.min_size - 1, p.min_size, p.min_size + 1, p.max_size,
              p.max_size + 1, L - 1, L, L + 1, 2 * L + 17, 5 * L + 4095):
        b = rng.integers(0, 256, n).astype(np.uint8)
        assert_same(gpu_chunk(gpu, b, p, seg=L), oracle.chunk(b, p))


def test_config1_random_16mib(gpu):
    """16 MiB of uniform random bytes (seed 0), 8 KiB preset, increasing."""
    b = W.uniform_random(16 << 20, 0)
    p = oracle.presets(8, 0)
    assert_same(gpu_chunk(gpu, b, p), oracle.chunk(b, p))


@pytest.mark.parametrize("seg", [4096, 16384, 65536, 262144])
@pytest.mark.parametrize("threads", [128, 256, 512])
def test_segment_and_block_size_invariance(gpu, seg, threads):
    b = W.mixed_base(8 << 20, 21)
    p = oracle.presets(8, 1)
    assert_same(gpu_chunk(gpu, b, p, seg=seg, threads=threads), oracle.chunk(b, p))


@pytest.mark.parametrize("pattern", ["zeros", "ramp", "saw3", "saw5", "saw9",
                                     "mixed_blocks"])
def test_adversarial_patterns(gpu, pattern):
    n = 3 << 20
    k = np.arange(n, dtype=np.int64)
    if pattern == "zeros":
        b = np.zeros(n, np.uint8)
    elif pattern == "ramp":
        b = (k % 256).astype(np.uint8)
    elif pattern.startswith("saw"):
        per = int(pattern[3:])
        b = ((k % per) * (256 // per)).astype(np.uint8)
    else:
        b = np.concatenate([W.adversarial_block(i, 3, block=1 << 19) for i in range(6)])
    for kib in (8, 16):
        for mode in (0, 1):
            p = oracle.presets(kib, mode)
            assert_same(gpu_chunk(gpu, b, p, seg=65536), oracle.chunk(b, p))


def test_batch_small_files(gpu):
    rng = np.random.default_rng(9)
    sizes = np.concatenate([[0, 1, 5, 0], rng.integers(0, 300000, 300), [0]])
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    data = W.mixed_base(int(offs[-1]), 4, block=4096)
    for p in (oracle.presets(4), oracle.presets(16, 1), Params(0, 3, 7, 40, 100, 700)):
        cuts, co = gpu_batch(gpu, data, offs, p, seg=8192)
        ecuts, eco = oracle.chunk_batch(data, offs, p)
        assert_same(co, eco)
        assert_same(cuts, ecuts)


def test_batch_empty(gpu):
    data = np.empty(0, np.uint8)
    cuts, co = gpu_batch(gpu, data, [0, 0, 0], oracle.presets(8))
    assert cuts.size == 0 and co.tolist() == [0, 0, 0]


@pytest.mark.slow
def test_config2_backup_stream_all_presets(gpu):
    """1 GiB backup-like stream; both modes at the 4, 8 and 16 KiB settings."""
    import torch
    from paper_2505_21194_gb300 import seqcdc as s
    data, _ = W.backup_stream(seed=0)
    d = torch.from_numpy(data).cuda()
    for kib in (4, 8, 16):
        for mode in (0, 1):
            p = oracle.presets(kib, mode)
            got = s.chunk(d, _p(s, p)).cpu().numpy().astype(np.uint64)
            assert_same(got, oracle.chunk(data, p))


@pytest.mark.slow
def test_config3_batched_10k_files(gpu):
    """10,000 log-normal files (median 256 KiB, sigma 1.5), CSR, 8 KiB preset."""
    data, offs = W.file_batch(10000, seed=0)
    p = oracle.presets(8, 0)
    cuts, co = gpu_batch(gpu, data, offs, p)
    ecuts, eco = oracle.chunk_batch_threaded(data, offs, p, os.cpu_count() or 4)
    assert_same(co, eco)
    assert_same(cuts, ecuts)


@pytest.mark.slow
def test_single_stream_beyond_4gib(gpu):
    """Offsets past 2^32 in one stream: 4 GiB + 64 KiB of zeros, then 16 MiB of
    random bytes.  Zeros hold no run, so every chunk there is cut at max_size
    (Sec. VI); the tail is checked against the oracle restarted at the last
    cut before it."""
    import torch
    s = gpu
    p = oracle.presets(16)
    zeros = (4 << 30) + (64 << 10)
    tail = W.uniform_random(16 << 20, 77)
    n = zeros + tail.size
    d = torch.zeros(n, dtype=torch.uint8, device="cuda")
    d[zeros:].copy_(torch.from_numpy(tail))
    got = s.chunk(d, _p(s, p)).cpu().numpy().astype(np.int64)
    del d
    torch.cuda.empty_cache()
    mx = p.max_size
    head = got[got <= zeros]
    assert np.array_equal(head, np.arange(1, head.size + 1, dtype=np.int64) * mx)
    start = int(head[-1])
    window = np.concatenate([np.zeros(zeros - start, np.uint8), tail])
    exp = oracle.chunk(window, p).astype(np.int64) + start
    assert np.array_equal(got[head.size:], exp)
