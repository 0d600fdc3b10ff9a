"""seqcdc_chunk_noalloc: the entry point for callers that cannot allocate.

Some callers may not call cudaMalloc: code hosted inside a process whose
device memory belongs to another allocator or pool, and latency-bound paths
where an allocation's implicit synchronisation is not acceptable.  For them
the library offers one entry point whose workspace is a fixed device array
compiled into the library.  This file checks, through the C ABI, that its cut
lists equal those of the allocating entry point (seqcdc_chunk), exactly, on
two calls in a row that reuse the shared array, and that inputs too large for
the array are refused.  It is named so that pytest collects it last.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2505_21194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _reference_cuts(s, d, p):
    """Cut list from the allocating entry point (caller-owned workspace)."""
    return s.chunk(d, p).cpu().numpy().astype(np.uint64)


def _noalloc_cuts(s, d, p):
    import torch
    n = d.numel()
    cap = n // p.min_size + 1
    cuts = torch.empty(max(cap, 1), dtype=torch.int64, device=d.device)
    count = torch.zeros(1, dtype=torch.int64, device=d.device)
    status = torch.full((1,), 99, dtype=torch.int32, device=d.device)
    s.seqcdc_chunk_noalloc(p, d, n, cuts, cap, count, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0, "device status %d" % int(status.item())
    return cuts[: int(count.item())].cpu().numpy().astype(np.uint64)


def test_noalloc_matches_allocating_entry_point_twice(gpu):
    import torch
    s = gpu
    cases = [
        (W.uniform_random(8 << 20, 31), s.seqcdc_params(8, 0)),
        (W.mixed_base(12 << 20, 32), s.seqcdc_params(16, 1)),
    ]
    for data, p in cases:  # two calls in a row share the fixed scratch
        d = torch.from_numpy(data).cuda()
        got = _noalloc_cuts(s, d, p)
        exp = _reference_cuts(s, d, p)
        assert got.size == exp.size and np.array_equal(got, exp)


def test_noalloc_refuses_inputs_beyond_its_scratch(gpu):
    s = gpu
    p = s.seqcdc_params(8, 0)
    n = 64 << 30  # far more than the fixed scratch can plan for, on either path
    for algo in (s.ALGO_MAP, s.ALGO_WALK):
        assert s.seqcdc_workspace_size(p, n, 1, (0, 0, algo, 0)) > s.SEQCDC_NOALLOC_SCRATCH_BYTES
    lib = s.load_library()
    import ctypes
    rc = lib.seqcdc_chunk_noalloc(ctypes.byref(p), 1 << 40, n, 1 << 40, n, 1 << 40,
                                  None, None, None)
    assert rc == s.SEQCDC_ERANGE
