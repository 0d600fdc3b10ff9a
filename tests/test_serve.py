"""Serving: the batching rule and statistics on the CPU; the server on the GPU.

On the GPU, every request of a short open-loop run is checked: its cut list
from the batch it was served in (a device tensor) must equal the oracle's for
its payload and the library's cut list for the payload chunked alone
(tolerance 0); a second run checks that serving allocates no device memory.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2505_21194_gb300 import workloads as W
from paper_2505_21194_gb300.serve import (Request, form_batch, latency_stats,
                                          poisson_arrivals)


def _reqs(sizes):
    return [Request(i, i, s, float(i)) for i, s in enumerate(sizes)]


def test_form_batch_fifo_and_limits():
    q = _reqs([10, 20, 30, 40])
    assert form_batch(q, 0, budget=1000, max_batch_bytes=1000) == 4
    assert form_batch(q, 0, budget=1000, max_batch_bytes=60) == 3     # 10+20+30
    assert form_batch(q, 0, budget=1000, max_batch_bytes=5) == 1      # head alone
    assert form_batch(q, 950, budget=1000, max_batch_bytes=1000) == 2  # 10+20 fit
    assert form_batch(q, 995, budget=1000, max_batch_bytes=1000) == 0  # head does not fit
    assert form_batch(_reqs([5, 500, 5]), 0, budget=100, max_batch_bytes=1000) == 1
    assert form_batch([], 0, 10, 10) == 0
    assert form_batch(q, 0, budget=1000, max_batch_bytes=1000, max_files=2) == 2
    assert form_batch(q, 0, budget=1000, max_batch_bytes=1000, max_files=1) == 1


def test_latency_stats_percentiles():
    lat = [i / 1000.0 for i in range(1, 101)]          # 1..100 ms
    s = latency_stats(lat)
    assert s["p50_ms"] == pytest.approx(50.5)
    assert s["p99_ms"] == pytest.approx(99.01)
    assert s["max_ms"] == pytest.approx(100.0)
    assert latency_stats([])["p50_ms"] is None


def test_poisson_arrivals_rate_and_order():
    sizes = [100, 200, 300]
    a = poisson_arrivals(2000.0, 5.0, 3, sizes, seed=1)
    assert abs(len(a) - 10000) < 400                   # 5 s at 2000/s
    t = np.array([r.arrival for r in a])
    assert (np.diff(t) > 0).all() and t[-1] <= 5.0
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1 / 2000.0, rel=0.05)
    assert all(r.nbytes == sizes[r.payload] for r in a)
    assert [r.rid for r in a] == list(range(len(a)))


@pytest.mark.gpu
def test_server_results_equal_oracle_and_alone(gpu):
    import torch
    from paper_2505_21194_gb300.serve import Server
    s = gpu
    p = s.seqcdc_params(8, 0)
    op = oracle.presets(8)
    rng = np.random.default_rng(3)
    sizes = rng.integers(1, 3 << 20, 12)
    sizes[0] = 0
    payloads = [W.mixed_base(int(n), 100 + k, block=4096) for k, n in enumerate(sizes)]
    offs = np.zeros(len(payloads) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    pool = torch.from_numpy(np.concatenate(payloads)).pin_memory()
    srv = Server(p, pool, offs, budget_bytes=64 << 20, max_batch_bytes=16 << 20)
    arr = poisson_arrivals(400.0, 0.25, len(payloads), sizes, seed=4)
    st = srv.run(arr, keep={r.rid for r in arr})
    assert st.requests == len(arr) and st.bytes == sum(r.nbytes for r in arr)
    assert st.latency["p50_ms"] is not None and st.latency["p99_ms"] >= st.latency["p50_ms"]
    alone = {}
    for k, b in enumerate(payloads):
        exp = oracle.chunk(b, op).astype(np.int64)
        if b.size:
            got_alone = s.chunk(torch.from_numpy(b).cuda(), p).cpu().numpy()
            assert np.array_equal(got_alone, exp)
        alone[k] = exp
    for r in arr:
        got = st.results[r.rid]
        assert got.is_cuda                       # cut lists stay on the device
        assert np.array_equal(got.cpu().numpy(), alone[r.payload]), r
    # Serving allocates nothing per batch: every buffer is in a slot made when
    # the server was built, and kept cut lists go to one buffer made before
    # the run's clock starts (none with no request kept).
    torch.cuda.synchronize()
    before = torch.cuda.memory_stats()["allocation.all.allocated"]
    st2 = srv.run(poisson_arrivals(400.0, 0.25, len(payloads), sizes, seed=5))
    torch.cuda.synchronize()
    assert st2.batches > 0 and st2.results == {}
    assert torch.cuda.memory_stats()["allocation.all.allocated"] == before
