"""Host-side pieces of bench.py: the chain walk's algorithmic bytes (the bytes
its chunks scan) and the DRAM-traffic records it reads."""
from __future__ import annotations

import json
import os

import numpy as np

import bench


class _P:
    def __init__(self, min_size, seq_length):
        self.min_size = min_size
        self.seq_length = seq_length


def _spans_direct(cuts, co, p):
    skip = max(p.min_size - p.seq_length, 0)
    total = 0
    for f in range(len(co) - 1):
        prev = 0
        for c in cuts[co[f]:co[f + 1]]:
            total += max(int(c) - prev - skip, 0)
            prev = int(c)
    return total


def test_scan_span_bytes_matches_a_direct_sum():
    import torch
    rng = np.random.default_rng(4)
    p = _P(4096, 5)
    cuts, co = [], [0]
    for f in range(60):
        n = int(rng.integers(0, 12))          # files with no cut and one cut included
        sizes = rng.integers(1, 20000, n)
        cuts.extend(np.cumsum(sizes).tolist())
        co.append(len(cuts))
    d_cuts = torch.tensor(cuts + [0, 0], dtype=torch.int64)   # spare entries past ncuts
    d_co = torch.tensor(co, dtype=torch.int64)
    got = bench.scan_span_bytes(d_cuts, d_co, len(cuts), p)
    assert got == _spans_direct(cuts, co, p)
    assert bench.scan_span_bytes(torch.zeros(4, dtype=torch.int64),
                                 torch.zeros(3, dtype=torch.int64), 0, p) == 0


def test_kernel_sources_exist_and_records_are_current_or_ignored():
    for kernel, files in bench.KERNEL_SOURCES.items():
        for rel in files:
            assert os.path.exists(os.path.join(bench.ROOT, rel)), rel
        rec = bench._traffic_record(kernel)
        path = os.path.join(bench.ROOT, "profiles", "%s_traffic.json" % kernel)
        if rec is not None:      # a record is used only while its sources match
            with open(path) as f:
                assert json.load(f)["source_sha256"] == bench._source_hash(kernel)
            assert 0 < rec["dram_bytes_per_byte"] < 2


def test_source_hash_ignores_comments_but_not_code():
    """A traffic record stays valid across edits to comments alone, and no
    longer matches once the code itself changes."""
    src = ('// head\n#include <x.h>\n/* block\n comment */\nint a = 1;  // trailing\n'
           'const char *s = "not // a comment";\nchar c = \'/\';\n\n')
    stripped = bench._strip_comments(src)
    assert stripped == ('#include <x.h>\nint a = 1;\nconst char *s = "not // a comment";\n'
                        "char c = '/';")
    reworded = src.replace("// trailing", "// reworded").replace("block", "other")
    assert bench._strip_comments(reworded) == stripped
    assert bench._strip_comments(src.replace("a = 1", "a = 2")) != stripped
