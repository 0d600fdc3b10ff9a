"""C ABI checks that need no GPU: the library builds, loads and exports every
entry point declared in include/seqcdc.h; host-side argument validation."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

import oracle

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "seqcdc.h")


def _declared():
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^[a-z0-9_ ]+\*?\s*(seqcdc_\w+)\(", text, re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("seqcdc_params", "seqcdc_chunk", "seqcdc_chunk_batch",
              "seqcdc_workspace_size", "seqcdc_status", "seqcdc_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(seqcdc_lib):
    lib = seqcdc_lib.load_library()
    for name in _declared():
        assert hasattr(lib, name), name


def test_presets_match_oracle(seqcdc_lib):
    for kib in (4, 8, 16):
        for mode in (0, 1):
            got = seqcdc_lib.seqcdc_params(kib, mode).astuple()
            o = oracle.presets(kib, mode)
            assert got == (o.mode, o.seq_length, o.skip_trigger, o.skip_size,
                           o.min_size, o.max_size)
    with pytest.raises(seqcdc_lib.SeqCDCError):
        seqcdc_lib.seqcdc_params(32, 0)
    with pytest.raises(seqcdc_lib.SeqCDCError):
        seqcdc_lib.seqcdc_params(8, 2)


@pytest.mark.parametrize("bad", [
    (2, 5, 50, 256, 4096, 16384),   # mode
    (0, 1, 50, 256, 4096, 16384),   # seq_length < 2
    (0, 17, 50, 256, 4096, 16384),  # seq_length > 16
    (0, 5, 50, 256, 0, 16384),      # min 0
    (0, 5, 50, 256, 8192, 4096),    # max < min
    (0, 5, 50, 256, 4096, 1 << 18), # max beyond the supported bound
])
def test_validate_rejects(seqcdc_lib, bad):
    p = seqcdc_lib.Params(*bad)
    assert seqcdc_lib.seqcdc_validate(p) == seqcdc_lib.SEQCDC_EINVAL
    lib = seqcdc_lib.load_library()
    assert lib.seqcdc_workspace_size(ctypes.byref(p), 1 << 20, 1, None) == 0


def test_workspace_size_grows(seqcdc_lib):
    s = seqcdc_lib
    p = s.seqcdc_params(8, 0)
    for algo in (s.ALGO_MAP, s.ALGO_WALK):
        t = (0, 0, algo, 0)
        a = s.seqcdc_workspace_size(p, 1 << 20, 1, t)
        b = s.seqcdc_workspace_size(p, 1 << 30, 1, t)
        c = s.seqcdc_workspace_size(p, 1 << 30, 10000, t)
        assert 0 < a < b < c


def test_host_side_errors_before_launch(seqcdc_lib):
    """Bad arguments are rejected on the host; nothing reaches the device."""
    lib = seqcdc_lib.load_library()
    p = seqcdc_lib.seqcdc_params(8, 0)
    P = ctypes.byref(p)
    n = 1 << 20
    ws = seqcdc_lib.seqcdc_workspace_size(p, n, 1)
    fake = 1 << 40  # never dereferenced: every call below fails validation
    E = seqcdc_lib
    # NULL / misaligned workspace
    assert lib.seqcdc_chunk(P, fake, n, fake, n, fake, None, ws, None, None) == E.SEQCDC_EINVAL
    assert lib.seqcdc_chunk(P, fake, n, fake, n, fake, fake + 8, ws, None, None) == E.SEQCDC_EINVAL
    # misaligned input
    assert lib.seqcdc_chunk(P, fake + 3, n, fake, n, fake, fake, ws, None, None) == E.SEQCDC_EINVAL
    # workspace too small (for either path), capacity too small
    ws_walk = seqcdc_lib.seqcdc_workspace_size(p, n, 1, (0, 0, E.ALGO_WALK, 0))
    assert ws_walk < ws
    assert lib.seqcdc_chunk(P, fake, n, fake, n, fake, fake, ws_walk - 1, None,
                            None) == E.SEQCDC_ECAPACITY
    t_map = ctypes.byref(E.Tuning(0, 0, E.ALGO_MAP, 0))
    assert lib.seqcdc_chunk(P, fake, n, fake, n, fake, fake, ws - 1, t_map,
                            None) == E.SEQCDC_ECAPACITY
    assert lib.seqcdc_chunk(P, fake, n, fake, n // 4096, fake, fake, ws, None, None) == E.SEQCDC_ECAPACITY
    # NULL count / offsets
    assert lib.seqcdc_chunk(P, fake, n, fake, n, None, fake, ws, None, None) == E.SEQCDC_EINVAL
    assert lib.seqcdc_chunk_batch(P, fake, n, None, 1, fake, n, fake, fake, ws, None, None) == E.SEQCDC_EINVAL
    bad = E.Params(0, 1, 0, 0, 1, 1)
    assert lib.seqcdc_chunk(ctypes.byref(bad), fake, n, fake, n, fake, fake, ws, None, None) == E.SEQCDC_EINVAL
    # range copies: NULL arrays or pointers with ranges to copy; nothing to copy is fine
    assert lib.seqcdc_copy_ranges(fake, fake, None, None, None, 3, None) == E.SEQCDC_EINVAL
    assert lib.seqcdc_copy_ranges(None, None, None, None, None, 0, None) == E.SEQCDC_OK


def test_strerror(seqcdc_lib):
    for code in range(6):
        assert seqcdc_lib.seqcdc_strerror(code)
    assert "unknown" in seqcdc_lib.seqcdc_strerror(99)


def test_resolve_tuning_defaults_and_rules(seqcdc_lib):
    s = seqcdc_lib
    for kib in (4, 8, 16):
        t = s.seqcdc_resolve_tuning(s.seqcdc_params(kib, 0))
        assert (t.segment_bytes, t.block_threads) == (65536, 256)
    p = s.seqcdc_params(8, 0)
    t = s.seqcdc_resolve_tuning(p, (4096, 128))      # raised to max_size
    assert (t.segment_bytes, t.block_threads) == (16384, 128)
    t = s.seqcdc_resolve_tuning(p, (70000, 300))     # 1 KiB multiple; default threads
    assert (t.segment_bytes, t.block_threads) == (70656, 256)
    t = s.seqcdc_resolve_tuning(p, (1 << 22, 256))   # capped at 1 MiB, then by smem
    assert t.segment_bytes <= 1 << 20 and t.segment_bytes % 1024 == 0
    with pytest.raises(s.SeqCDCError):
        s.seqcdc_resolve_tuning(s.Params(2, 5, 50, 256, 4096, 16384))


def test_resolve_tuning_piece_rules(seqcdc_lib):
    """Chain-walk piece size: default 768 KiB (384 x min_size above a 4 KiB
    minimum); rounded up to 64 KiB; at least
    4 x max_size; at most 64 MiB.  The algorithm field is passed through."""
    s = seqcdc_lib
    p8, p16 = s.seqcdc_params(8, 0), s.seqcdc_params(16, 0)
    t = s.seqcdc_resolve_tuning(p8)
    assert t.piece_bytes == 768 << 10 and t.algorithm == s.ALGO_AUTO
    t = s.seqcdc_resolve_tuning(p8, (0, 0, s.ALGO_WALK, 100000))
    assert t.piece_bytes == 131072 and t.algorithm == s.ALGO_WALK
    assert s.seqcdc_resolve_tuning(p8, (0, 0, 2, 65536)).piece_bytes == 65536
    assert s.seqcdc_resolve_tuning(p16, (0, 0, 2, 65536)).piece_bytes == 131072
    assert s.seqcdc_resolve_tuning(p8, (0, 0, 2, 1 << 30)).piece_bytes == 64 << 20
    assert s.seqcdc_resolve_tuning(p8, (0, 0, s.ALGO_MAP, 0)).algorithm == s.ALGO_MAP
    # the default grows with min_size above 4 KiB (16 KB setting: min 8 KiB)
    assert s.seqcdc_resolve_tuning(s.seqcdc_params(4, 0)).piece_bytes == 768 << 10
    assert s.seqcdc_resolve_tuning(p16).piece_bytes == 384 * 8192
    assert s.seqcdc_resolve_tuning(p16, (0, 0, 2, 1 << 20)).piece_bytes == 1 << 20


def test_workspace_follows_the_path(seqcdc_lib):
    """A batch of at least SEQCDC_WALK_MIN_FILES files, or of at least
    SEQCDC_WALK_MIN_PIECES full pieces, takes the chain walk by default and
    sizes its workspace for it; forcing either path sizes for that path; a
    short single stream takes the segment map."""
    s = seqcdc_lib
    p = s.seqcdc_params(8, 0)
    total, many, few = 8 << 30, s.WALK_MIN_FILES, s.WALK_MIN_FILES - 1
    walk = s.seqcdc_workspace_size(p, total, many, (0, 0, s.ALGO_WALK, 0))
    smap = s.seqcdc_workspace_size(p, total, many, (0, 0, s.ALGO_MAP, 0))
    assert walk < smap
    assert s.seqcdc_workspace_size(p, total, many) == walk
    # few files but many pieces: still the walk; few files of few pieces: the map
    assert s.seqcdc_workspace_size(p, total, few) == \
        s.seqcdc_workspace_size(p, total, few, (0, 0, s.ALGO_WALK, 0))
    small = (s.WALK_MIN_PIECES - 1) * (768 << 10)
    assert s.seqcdc_workspace_size(p, small, few) == \
        s.seqcdc_workspace_size(p, small, few, (0, 0, s.ALGO_MAP, 0))
    big = ws = 1 << 62
    for t, nf, batch, algo in ((small, 1, False, s.ALGO_MAP),
                               (small + (768 << 10), 1, False, s.ALGO_WALK),
                               (small, few, True, s.ALGO_MAP),
                               (small, many, True, s.ALGO_WALK),
                               (total, 1, False, s.ALGO_WALK)):
        assert s.seqcdc_algorithm(p, t, nf, batch, ws) == algo, (t, nf, batch)
    assert s.seqcdc_algorithm(p, total, 1, False, big, (0, 0, s.ALGO_MAP, 0)) == s.ALGO_MAP
    # 8 GiB in 768 KiB pieces: the walk's lists take a few bytes per input KiB
    assert walk < total // 64


def test_walk_workspace_is_monotone(seqcdc_lib):
    """The chain walk's workspace grows with the bytes and the files, so a
    workspace sized for a batch serves every smaller one (what AUTO's
    fallback to the walk relies on)."""
    s = seqcdc_lib
    rng = np.random.default_rng(0)
    for kib in (4, 8, 16):
        p = s.seqcdc_params(kib, 0)
        t = (0, 0, s.ALGO_WALK, 0)
        for _ in range(200):
            t1 = int(rng.integers(0, 1 << 34))
            f1 = int(rng.integers(1, 20000))
            t2 = t1 + int(rng.integers(0, 1 << 30))
            f2 = f1 + int(rng.integers(0, 5000))
            assert s.seqcdc_workspace_size(p, t1, f1, t) <= s.seqcdc_workspace_size(p, t2, f2, t)


@pytest.mark.gpu
def test_chunk_batch_in_a_cuda_graph_with_profile_events(gpu):
    """The batched call captured into a CUDA graph (as bench.py times it):
    replays give the direct call's cut list, and the measurement events,
    recorded as external event nodes during capture, bracket the dominant
    kernel on every replay."""
    import torch
    from paper_2505_21194_gb300 import workloads as W
    s = gpu
    data, offs = W.file_batch(300, seed=4)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(offs.astype(np.int64)).cuda()
    p = s.seqcdc_params(8, 0)
    ref = s.chunk_batch(d, o, p)
    nf, total = o.numel() - 1, d.numel()
    cap = total // p.min_size + nf
    cuts = torch.full((cap,), -1, dtype=torch.int64, device="cuda")
    co = torch.empty(nf + 1, dtype=torch.int64, device="cuda")
    ws_bytes = s.seqcdc_workspace_size(p, total, nf)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for e in evs:
        e.record()
    gs = torch.cuda.Stream()
    gs.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(gs):
        s.seqcdc_chunk_batch(p, d, total, o, nf, cuts, cap, co, ws, ws_bytes, None, gs)
        gs.synchronize()
        with torch.cuda.graph(graph, stream=gs):
            for i in range(2):
                s.seqcdc_profile_events(evs[2 * i], evs[2 * i + 1])
                s.seqcdc_chunk_batch(p, d, total, o, nf, cuts, cap, co, ws, ws_bytes, None, gs)
        s.seqcdc_profile_events(None, None)
    torch.cuda.current_stream().wait_stream(gs)
    for _ in range(2):
        cuts.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        assert s.seqcdc_status(ws) == s.SEQCDC_OK
        k = int(co[-1].item())
        assert np.array_equal(co.cpu().numpy(), ref.cut_offsets.cpu().numpy())
        assert np.array_equal(cuts[:k].cpu().numpy(), ref.cuts.cpu().numpy())
        for i in range(2):
            assert evs[2 * i].elapsed_time(evs[2 * i + 1]) > 0.0


@pytest.mark.gpu
def test_copy_ranges_gathers_host_and_device_ranges(gpu):
    """seqcdc_copy_ranges: ranges of a pinned host buffer gathered into a
    device buffer in any order, including empty ranges, and back."""
    import numpy as np
    import torch
    s = gpu
    rng = np.random.default_rng(3)
    pool = torch.from_numpy(rng.integers(0, 256, 1 << 20, dtype=np.uint8)).pin_memory()
    lens = np.array([100, 0, 4096, 7, 65536, 1], dtype=np.uint64)
    src = np.array([5, 17, 1000, 999_990, 200_000, 0], dtype=np.uint64)
    dst = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.uint64)
    d = torch.zeros(int(lens.sum()), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    s.seqcdc_copy_ranges(d, pool, dst, src, lens, st)
    back = torch.zeros(int(lens.sum()), dtype=torch.uint8).pin_memory()
    s.seqcdc_copy_ranges(back, d, [0], [0], [int(lens.sum())], st)
    st.synchronize()
    want = np.concatenate([pool.numpy()[a:a + n] for a, n in zip(src.tolist(), lens.tolist())])
    assert np.array_equal(back.numpy(), want)
