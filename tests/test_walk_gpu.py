"""GPU parity of the chain-walking path against the CPU oracle.

The chain walk follows the chunk chain of every piece with one warp, joins
pieces with junction walks and repairs pieces whose junction started from a
wrong exit.  These cases force that path (algorithm = ALGO_WALK) with the
smallest pieces the parameters allow, so that junctions that meet, junctions
that leave their piece, and the repair pass all run; results must equal the
oracle's cut lists exactly.  The counters of seqcdc_stats show which of those
code paths ran.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2505_21194_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WALK = 2
MAP = 1


def _p(s, p: Params):
    return s.make_params(p.mode, p.seq_length, p.skip_trigger, p.skip_size,
                         p.min_size, p.max_size)


def walk_chunk(s, b, p: Params, piece=0):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    return s.chunk(d, _p(s, p), tuning=(0, 0, WALK, piece)).cpu().numpy().astype(np.uint64)


def walk_batch(s, data, offs, p: Params, piece=0, algorithm=WALK):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    o = torch.from_numpy(np.asarray(offs, dtype=np.int64)).cuda()
    r = s.chunk_batch(d, o, _p(s, p), tuning=(0, 0, algorithm, piece))
    return r.cuts.cpu().numpy().astype(np.uint64), r.cut_offsets.cpu().numpy().astype(np.uint64)


def walk_stats(s, data, offs, p: Params, piece=0):
    """Chunk a batch with the chain walk and return its path counters."""
    import torch
    d = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    o = torch.from_numpy(np.asarray(offs, dtype=np.int64)).cuda()
    pp = _p(s, p)
    t = (0, 0, WALK, piece)
    nfiles = len(offs) - 1
    total = int(offs[-1])
    ws_bytes = s.seqcdc_workspace_size(pp, total, nfiles, t)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    cap = total // pp.min_size + nfiles
    cuts = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    co = torch.empty(nfiles + 1, dtype=torch.int64, device="cuda")
    s.seqcdc_chunk_batch(pp, d, total, o, nfiles, cuts, cap, co, ws, ws_bytes, t)
    assert s.seqcdc_status(ws) == 0
    st = list(s.seqcdc_stats(ws).values())
    n = int(co[-1].item())
    return st, cuts[:n].cpu().numpy().astype(np.uint64), co.cpu().numpy().astype(np.uint64)


def same(got, exp):
    got = np.asarray(got, np.uint64)
    exp = np.asarray(exp, np.uint64)
    assert got.size == exp.size, (got.size, exp.size)
    if not np.array_equal(got, exp):
        k = int(np.argmax(got != exp))
        raise AssertionError("first difference at %d: gpu %s oracle %s" % (
            k, got[k:k + 4].tolist(), exp[k:k + 4].tolist()))


@pytest.mark.parametrize("seed", range(24))
def test_walk_random_streams(gpu, seed):
    """Random parameter sets (SeqLength 2..16, BASE, small skips, min 1) on
    random, small-alphabet, text and mixed inputs, one stream each."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(0, 600000))
    kind = seed % 4
    if kind == 0:
        b = rng.integers(0, 256, n).astype(np.uint8)
    elif kind == 1:
        b = rng.integers(0, 3, n).astype(np.uint8)
    elif kind == 2:
        b = W.markov_text(n, seed)
    else:
        b = W.mixed_base(n, seed, block=8192) if n else np.empty(0, np.uint8)
    R = int(rng.choice([2, 3, 5, 8, 16]))
    mn = int(rng.integers(1, 5000))
    mx = int(rng.integers(mn, min(mn + 12000, 16384) + 1))
    p = Params(int(rng.integers(0, 2)), R, int(rng.choice([0, 1, 7, 50])),
               int(rng.integers(0, 700)), mn, mx)
    same(walk_chunk(gpu, b, p, piece=65536), oracle.chunk(b, p))


@pytest.mark.parametrize("kib", [4, 8, 16])
@pytest.mark.parametrize("mode", [0, 1])
def test_walk_presets_edge_lengths(gpu, kib, mode):
    p = oracle.presets(kib, mode)
    rng = np.random.default_rng(kib * 10 + mode + 500)
    P = max(65536, 4 * p.max_size)
    for n in (0, 1, 2, p.min_size - 1, p.min_size, p.min_size + 1, p.max_size,
              p.max_size + 1, P - 1, P, P + 1, 2 * P + 17, 5 * P + 4095):
        b = rng.integers(0, 256, n).astype(np.uint8)
        same(walk_chunk(gpu, b, p, piece=P), oracle.chunk(b, p))


@pytest.mark.parametrize("pattern", ["zeros_after_random", "ramp", "saw3", "saw5",
                                     "mixed_blocks"])
def test_walk_adversarial(gpu, pattern):
    """Stretches where chains started at different places never meet: every
    piece's junction leaves the piece and the repair pass walks them."""
    n = 3 << 20
    k = np.arange(n, dtype=np.int64)
    rng = np.random.default_rng(77)
    if pattern == "zeros_after_random":
        b = np.zeros(n, np.uint8)
        b[:6000] = rng.integers(0, 256, 6000)
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
            same(walk_chunk(gpu, b, p, piece=4 * p.max_size), oracle.chunk(b, p))


def test_walk_repair_path_runs(gpu):
    """A batch whose files start with a few random bytes and continue with
    zeros: chains are offset from the piece starts, so junctions cannot meet
    and the repair pass must redo them.  Exact output and non-zero counters."""
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in rng.integers(300000, 900000, 260)]
    parts = []
    for s_ in sizes:
        f = np.zeros(s_, np.uint8)
        f[:6000] = rng.integers(0, 256, 6000)
        parts.append(f)
    data = np.concatenate(parts)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    p = oracle.presets(8)
    st, cuts, co = walk_stats(gpu, data, offs, p, piece=65536)
    ecuts, eco = oracle.chunk_batch(data, offs, p)
    same(co, eco)
    same(cuts, ecuts)
    assert st[2] > 0 and st[4] > 0 and st[5] > 0 and st[6] > 0, st


def test_walk_batch_small_files(gpu):
    rng = np.random.default_rng(9)
    sizes = np.concatenate([[0, 1, 5, 0], rng.integers(0, 300000, 300), [0]])
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    data = W.mixed_base(int(offs[-1]), 4, block=4096)
    for p in (oracle.presets(4), oracle.presets(16, 1), Params(0, 3, 7, 40, 100, 700)):
        for piece in (0, 65536):
            cuts, co = walk_batch(gpu, data, offs, p, piece=piece)
            ecuts, eco = oracle.chunk_batch(data, offs, p)
            same(co, eco)
            same(cuts, ecuts)


def test_walk_batch_empty_and_tiny(gpu):
    cuts, co = walk_batch(gpu, np.empty(0, np.uint8), [0, 0, 0], oracle.presets(8))
    assert cuts.size == 0 and co.tolist() == [0, 0, 0]
    data = np.arange(7, dtype=np.uint8)
    cuts, co = walk_batch(gpu, data, [0, 0, 3, 3, 7], oracle.presets(8))
    assert co.tolist() == [0, 0, 1, 1, 2] and cuts.tolist() == [3, 4]


def test_walk_and_map_agree_on_mixed_batch(gpu):
    """Both paths on the same 1,000-file batch (log-normal sizes): identical
    output, equal to the oracle."""
    data, offs = W.file_batch(1000, seed=3, median=64 << 10)
    p = oracle.presets(8, 1)
    c_w, o_w = walk_batch(gpu, data, offs, p, algorithm=WALK)
    c_m, o_m = walk_batch(gpu, data, offs, p, algorithm=MAP)
    same(o_w, o_m)
    same(c_w, c_m)
    ecuts, eco = oracle.chunk_batch(data, offs, p)
    same(o_w, eco)
    same(c_w, ecuts)


@pytest.mark.slow
def test_walk_config3_full_size(gpu):
    """10,000 log-normal files (median 256 KiB, sigma 1.5), 8 KiB preset, in
    the benchmark's launch configuration (default tuning: the chain walk)."""
    import os
    data, offs = W.file_batch(10000, seed=0)
    p = oracle.presets(8, 0)
    cuts, co = walk_batch(gpu, data, offs, p, algorithm=0)
    ecuts, eco = oracle.chunk_batch_threaded(data, offs, p, os.cpu_count() or 4)
    same(co, eco)
    same(cuts, ecuts)


@pytest.mark.slow
def test_walk_offsets_beyond_4gib(gpu):
    """One stream of 4 GiB + 64 KiB of zeros and 16 MiB of random bytes with
    the chain walk: forced cuts every max_size, then the oracle's cuts of the
    tail restarted at the last forced cut."""
    import torch
    s = gpu
    p = oracle.presets(16)
    zeros = (4 << 30) + (64 << 10)
    tail = W.uniform_random(16 << 20, 78)
    n = zeros + tail.size
    d = torch.zeros(n, dtype=torch.uint8, device="cuda")
    d[zeros:].copy_(torch.from_numpy(tail))
    got = s.chunk(d, _p(s, p), tuning=(0, 0, WALK, 0)).cpu().numpy().astype(np.int64)
    del d
    torch.cuda.empty_cache()
    mx = p.max_size
    head = got[got <= zeros]
    assert np.array_equal(head, np.arange(1, head.size + 1, dtype=np.int64) * mx)
    start = int(head[-1])
    window = np.concatenate([np.zeros(zeros - start, np.uint8), tail])
    exp = oracle.chunk(window, p).astype(np.int64) + start
    assert np.array_equal(got[head.size:], exp)


def test_auto_workspace_sized_for_a_larger_batch(gpu):
    """A workspace sized for 300 files (the chain walk under AUTO) serves a
    call with 200 of them, which AUTO alone would give the segment map with
    its larger workspace: the call takes the chain walk and is exact."""
    import torch
    s = gpu
    p = oracle.presets(8)
    pp = _p(s, p)
    rng = np.random.default_rng(12)
    sizes = rng.integers(1000, 200000, 300)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    data = W.mixed_base(int(offs[-1]), 6, block=4096)
    ws_bytes = s.seqcdc_workspace_size(pp, int(offs[-1]), 300)
    assert ws_bytes < s.seqcdc_workspace_size(pp, int(offs[200]), 200)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    sub = offs[:201]
    total = int(sub[-1])
    d = torch.from_numpy(data[:total]).cuda()
    o = torch.from_numpy(sub).cuda()
    cap = total // pp.min_size + 200
    cuts = torch.empty(cap, dtype=torch.int64, device="cuda")
    co = torch.empty(201, dtype=torch.int64, device="cuda")
    s.seqcdc_chunk_batch(pp, d, total, o, 200, cuts, cap, co, ws, ws_bytes)
    assert s.seqcdc_status(ws) == 0
    n = int(co[-1].item())
    ecuts, eco = oracle.chunk_batch(data[:total], sub.astype(np.uint64), p)
    same(co.cpu().numpy(), eco)
    same(cuts[:n].cpu().numpy(), ecuts)
