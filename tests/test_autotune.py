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
    assert c and all(L >= p.max_size for L, _ in c)
    assert {t for _, t in c} == {128, 256, 512}
    for L, t in c:
        e = s.seqcdc_resolve_tuning(p, (L, t))
        assert (e.segment_bytes, e.block_threads) == (L, t)
    p4 = s.seqcdc_params(4, 0)
    assert (32768, 256) in A.candidates(p4)


def test_workload_key_separates_shapes(seqcdc_lib):
    p = seqcdc_lib.seqcdc_params(8, 0)
    k1 = A.workload_key("GPU", 152, p, [1 << 20])
    k2 = A.workload_key("GPU", 152, p, [1 << 18] * 9)
    k3 = A.workload_key("GPU", 148, p, [1 << 20])
    k4 = A.workload_key("GPU", 152, seqcdc_lib.seqcdc_params(8, 1), [1 << 20])
    assert len({k1, k2, k3, k4}) == 4
    assert A.workload_key("GPU", 152, p, [300000] * 5) == A.workload_key("GPU", 152, p, [270000] * 7)


def test_pick_best_and_ties():
    t = {(65536, 256): 2.0, (32768, 128): 1.5, (131072, 512): 1.5}
    assert A.pick_best(t) == (32768, 128)
    assert A.pick_best(t, default=(65536, 256)) == (32768, 128)     # default too slow
    t2 = {(65536, 256): 1.005, (131072, 512): 1.0, (32768, 128): 1.3}
    assert A.pick_best(t2, default=(65536, 256)) == (65536, 256)    # within 1 %
    assert A.pick_best(t2) == (65536, 256)                          # smaller segment
    assert A.pick_best(t2, tol=0.0) == (131072, 512)


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "sub" / "tuning.json")
    assert A.load_cache(path) == {}
    A.store_cache(path, "k1", {"segment_bytes": 65536, "block_threads": 256})
    A.store_cache(path, "k2", {"segment_bytes": 131072, "block_threads": 512})
    d = json.load(open(path))
    assert d["k1"]["segment_bytes"] == 65536 and d["k2"]["block_threads"] == 512
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
    cands = [(65536, 256), (131072, 512), (32768, 128)]
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
