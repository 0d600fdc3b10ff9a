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
from paper_2505_21194_gb300.serve import (Cancellations, Request, form_batch, latency_stats,
                                          poisson_arrivals, withdraw)


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


def test_withdraw_keeps_order():
    import collections
    q = collections.deque(_reqs([1, 2, 3, 4, 5]))
    assert withdraw(q, {1, 3, 9}) == 2
    assert [r.rid for r in q] == [0, 2, 4]
    assert withdraw(q, set()) == 0 and len(q) == 3


def test_cancellations_in_a_simulated_serving_loop():
    """The serving loop's order on a host-only model of the device
    (arrivals join the queue, cancellations are applied, finished batches
    leave, the next batch is admitted; one batch in flight, each taking a
    fixed time): every request is either served once or cancelled, never
    both; a cancelled request was never admitted and its time had come; a
    served request with a cancellation was admitted before it."""
    import collections
    rng = np.random.default_rng(5)
    sizes = rng.integers(1, 100, 400)
    arrivals = poisson_arrivals(2000.0, 0.2, len(sizes), sizes, seed=6)
    cancels = {r.rid: r.arrival + float(rng.uniform(-0.002, 0.01))
               for r in arrivals if rng.random() < 0.3}
    cancels[10 ** 6] = 0.05            # an id that never arrives changes nothing
    cancel = Cancellations(cancels)
    queue, admitted_at, served = collections.deque(), {}, []
    i, now, busy_until, inflight = 0, 0.0, -1.0, []
    removed_at = {}
    while i < len(arrivals) or queue or inflight:
        while i < len(arrivals) and arrivals[i].arrival <= now:
            queue.append(arrivals[i])
            i += 1
        before = {r.rid for r in queue}
        cancel.tick(now, queue, i)
        for rid in before - {r.rid for r in queue}:
            removed_at[rid] = now
        if inflight and now >= busy_until:
            served += inflight
            inflight = []
        if queue and not inflight:
            k = form_batch(queue, 0, budget=10 ** 9, max_batch_bytes=500)
            inflight = [queue.popleft() for _ in range(k)]
            for r in inflight:
                admitted_at[r.rid] = now
            busy_until = now + 0.003
        now = round(now + 0.0005, 7)
    served_ids = [r.rid for r in served]
    assert len(served_ids) == len(set(served_ids))
    assert set(served_ids).isdisjoint(removed_at)
    assert set(served_ids) | set(removed_at) == {r.rid for r in arrivals}
    for rid, t in removed_at.items():
        assert rid not in admitted_at and cancels[rid] <= t
    late = [rid for rid in served_ids if rid in cancels]
    assert all(admitted_at[rid] < cancels[rid] for rid in late)
    assert cancel.cancelled == len(removed_at) > 0
    assert cancel.too_late(arrivals) == len(late) > 0
    assert not Cancellations(None) and not Cancellations({})


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


@pytest.mark.gpu
def test_server_cancellations(gpu):
    """Requests whose client cancels them before the run starts are never
    chunked and have no result; requests cancelled only after the run ends
    were admitted first, so they are served (cut lists equal to the
    oracle's) and their cancellations are counted as too late."""
    import torch
    from paper_2505_21194_gb300.serve import Server
    s = gpu
    p = s.seqcdc_params(8, 0)
    op = oracle.presets(8)
    rng = np.random.default_rng(8)
    sizes = rng.integers(1, 2 << 20, 8)
    payloads = [W.mixed_base(int(n), 200 + k, block=4096) for k, n in enumerate(sizes)]
    offs = np.zeros(len(payloads) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    pool = torch.from_numpy(np.concatenate(payloads)).pin_memory()
    srv = Server(p, pool, offs, budget_bytes=64 << 20, max_batch_bytes=16 << 20)
    arr = poisson_arrivals(400.0, 0.1, len(payloads), sizes, seed=9)
    early = {r.rid for r in arr[::3]}
    late = {r.rid for r in arr[1::3]}
    assert early and late
    cancels = {rid: -1.0 for rid in early}
    cancels.update({rid: 1e9 for rid in late})
    st = srv.run(arr, keep={r.rid for r in arr}, cancels=cancels)
    assert st.cancelled == len(early) and st.cancel_too_late == len(late)
    assert st.requests == len(arr) - len(early)
    assert st.bytes == sum(r.nbytes for r in arr if r.rid not in early)
    assert set(st.results) == {r.rid for r in arr} - early
    want = {k: oracle.chunk(b, op).astype(np.int64) for k, b in enumerate(payloads)}
    for r in arr:
        if r.rid not in early:
            assert np.array_equal(st.results[r.rid].cpu().numpy(), want[r.payload]), r
