"""Bounded device waits: a wait that runs out is reported, not hung on.

The segment map resolves each segment's true entry by decoupled look-back,
which waits for a preceding segment to publish its exit (the chunk chain of
Sec. III is sequential).  Every such wait is bounded; seqcdc_set_wait_limit_ns
sets the bound for the calling host thread.  The GPU test makes the waits run
out on purpose (a bound of 0 on input where every look-back has to wait) and
checks that the call returns at once with SEQCDC_ETIMEOUT in the device
status, and that the same context then chunks the same input exactly with the
default bound.  Nothing here faults, traps or hangs a GPU.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle


def test_wait_limit_setter_is_per_thread_and_returns_previous(seqcdc_lib):
    import threading
    s = seqcdc_lib
    assert s.DEFAULT_WAIT_NS == 2_000_000_000
    prev = s.seqcdc_set_wait_limit_ns(123)
    try:
        assert prev == s.DEFAULT_WAIT_NS
        seen = []
        t = threading.Thread(target=lambda: seen.append(s.seqcdc_set_wait_limit_ns(7)))
        t.start()
        t.join()
        assert seen == [s.DEFAULT_WAIT_NS]        # another thread: its own default
        assert s.seqcdc_set_wait_limit_ns(0) == 123
    finally:
        s.seqcdc_set_wait_limit_ns(s.DEFAULT_WAIT_NS)


@pytest.mark.gpu
def test_expired_wait_reports_timeout_and_context_stays_usable(gpu):
    import torch
    s = gpu
    p = s.seqcdc_params(8, 0)
    # Constant bytes have no run ends, so no segment has a natural cut: every
    # segment's exit is a forced cut that only its predecessor's true exit
    # decides, and every look-back must wait for it.  4096 segments of 64 KiB.
    n = 256 << 20
    d = torch.zeros(n, dtype=torch.uint8, device="cuda")
    tuning = s.Tuning(65536, 256, s.ALGO_MAP, 0)
    cap = n // p.min_size + 1
    cuts = torch.empty(cap, dtype=torch.int64, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    ws_bytes = s.seqcdc_workspace_size(p, n, 1, tuning)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    prev = s.seqcdc_set_wait_limit_ns(0)
    try:
        t0 = time.perf_counter()
        s.seqcdc_chunk(p, d, n, cuts, cap, count, ws, ws_bytes, tuning)
        status = s.seqcdc_status(ws)
        dt = time.perf_counter() - t0
    finally:
        assert s.seqcdc_set_wait_limit_ns(prev) == 0
    assert status == s.SEQCDC_ETIMEOUT
    assert dt < 1.0, dt     # far below one default bound (2 s) per wait
    # The context is still usable: the default bound gives the exact cuts.
    got = s.chunk(d, p, tuning).cpu().numpy().astype(np.uint64)
    exp = oracle.chunk(np.zeros(n, np.uint8), oracle.presets(8, 0))
    assert np.array_equal(got, exp)
    assert s.seqcdc_status(ws) == s.SEQCDC_ETIMEOUT   # the old workspace keeps its status
