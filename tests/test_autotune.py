"""Launch tuning: cache keys, candidates, choice and cache reuse."""
from __future__ import annotations

import json

import numpy as np
import pytest

from paper_2505_21194_gb300 import autotune as A


def test_candidates_respect_max_size_and_library_rules(seqcdc_lib):
    s = seqcdc_lib
    p = s.seqcdc_params(16, 0)                    # max_size 32 KiB
    c = A.candidates(p)
    maps = [x for x in c if x[2] == s.ALGO_MAP]
    walks = [x for x in c if x[2] == s.ALGO_WALK]
    assert maps and all(L >= p.max_size for L, _, _, _ in maps)
    assert {t for _, t, _, _ in maps} == {128, 256, 512}
    for L, t, a, P in maps:
        e = s.seqcdc_resolve_tuning(p, (L, t, a, P))
        assert (e.segment_bytes, e.block_threads) == (L, t)
    # pieces below 4 x max_size (128 KiB here) are not candidates
    assert walks and all(P >= 4 * p.max_size for _, _, _, P in walks)
    for x in walks:
        assert s.seqcdc_resolve_tuning(p, x).piece_bytes == x[3]
    p4 = s.seqcdc_params(4, 0)
    assert (32768, 256, s.ALGO_MAP, 0) in A.candidates(p4)
    assert (0, 0, s.ALGO_WALK, 262144) in A.candidates(p4)


def test_default_candidate_follows_auto_rule(seqcdc_lib):
    s = seqcdc_lib
    p = s.seqcdc_params(8, 0)
    assert A.default_candidate(p, s.WALK_MIN_FILES) == (0, 0, s.ALGO_WALK, 768 << 10)
    assert A.default_candidate(p, s.WALK_MIN_FILES - 1) == (65536, 256, s.ALGO_MAP, 0)
    assert A.default_candidate(p, 1000, batch=False)[2] == s.ALGO_MAP
    # a stream of at least SEQCDC_WALK_MIN_PIECES full pieces takes the walk
    assert A.default_candidate(p, 1, False, 2 << 30)[2] == s.ALGO_WALK
    assert A.default_candidate(p, 1, False, 256 << 20)[2] == s.ALGO_MAP


def test_workload_key_separates_shapes(seqcdc_lib):
    p = seqcdc_lib.seqcdc_params(8, 0)
    k1 = A.workload_key("GPU", 152, p, [1 << 20])
    k2 = A.workload_key("GPU", 152, p, [1 << 18] * 9)
    k3 = A.workload_key("GPU", 148, p, [1 << 20])
    k4 = A.workload_key("GPU", 152, seqcdc_lib.seqcdc_params(8, 1), [1 << 20])
    k5 = A.workload_key("GPU", 152, p, [1 << 18] * 900)
    assert len({k1, k2, k3, k4, k5}) == 5
    assert A.workload_key("GPU", 152, p, [300000] * 5) == A.workload_key("GPU", 152, p, [270000] * 7)
    assert A.workload_key("GPU", 152, p, [1 << 18]).startswith(A.CACHE_VERSION + "|")


def test_pick_best_and_ties():
    t = {(65536, 256): 2.0, (32768, 128): 1.5, (131072, 512): 1.5}
    w = {(65536, 256, 1, 0): 2.0, (0, 0, 2, 1 << 20): 1.0, (0, 0, 2, 1 << 19): 1.002}
    assert A.pick_best(w, default=(0, 0, 2, 1 << 20)) == (0, 0, 2, 1 << 20)
    assert A.pick_best(w) == (0, 0, 2, 1 << 19)
    assert A.pick_best(t) == (32768, 128)
    assert A.pick_best(t, default=(65536, 256)) == (32768, 128)     # default too slow
    t2 = {(65536, 256): 1.005, (131072, 512): 1.0, (32768, 128): 1.3}
    assert A.pick_best(t2, default=(65536, 256)) == (65536, 256)    # within 1 %
    assert A.pick_best(t2) == (65536, 256)                          # smaller segment
    assert A.pick_best(t2, tol=0.0) == (131072, 512)


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    assert A.load_cache(path) == {}
    A.store_cache(path, "k1", {"tuning": [65536, 256, 1, 0]})
    A.store_cache(path, "k2", {"tuning": [0, 0, 2, 1 << 20]})
    d = json.load(open(path))
    assert d["k1"]["tuning"] == [65536, 256, 1, 0] and d["k2"]["tuning"][3] == 1 << 20
    (tmp_path / "bad.json").write_text("not json")
    assert A.load_cache(str(tmp_path / "bad.json")) == {}


@pytest.mark.gpu
def test_autotune_times_once_then_hits_cache(gpu, tmp_path):
    import torch
    from paper_2505_21194_gb300 import workloads as W
    s = gpu
    p = s.seqcdc_params(8, 0)
    data, offs = W.file_batch(40, seed=2)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(offs.astype(np.int64)).cuda()
    path = str(tmp_path / "t.json")
    cands = [(65536, 256, 1, 0), (131072, 512, 1, 0), (0, 0, 2, 1 << 18)]
    calls = []

    def timer(p_, d_, o_, c):
        calls.append(c)
        return A.time_candidate(p_, d_, o_, c, reps=2, warmup=1)

    best = A.autotune(p, d, o, cache_path=path, cands=cands, timer=timer)
    assert best in cands and sorted(calls) == sorted(cands)
    calls.clear()
    assert A.autotune(p, d, o, cache_path=path, cands=cands, timer=timer) == best
    assert calls == []
    r = s.chunk_batch(d, o, p, tuning=best)
    assert int(r.cut_offsets[-1]) == r.cuts.numel()
