"""Parameter sweep: settings, and means equal to the oracle's on a sample."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import Params
from paper_2505_21194_gb300 import workloads as W


def test_table1_settings(seqcdc_lib):
    from paper_2505_21194_gb300.sweep import table1_settings
    a = table1_settings()
    assert [s[1:4] for s in a] == [(5, 55, 256), (5, 50, 256), (5, 50, 512)]
    assert [s[4:] for s in a] == [(1024, 8192), (4096, 16384), (8192, 32768)]
    assert [s[1] for s in table1_settings(extra_run_byte=True)] == [6, 6, 6]
    assert [s[2] for s in table1_settings(base=True)] == [0, 0, 0]


@pytest.mark.gpu
def test_sweep_means_equal_oracle(gpu):
    import torch
    from paper_2505_21194_gb300.sweep import sweep, table1_settings
    data = W.mixed_base(8 << 20, 11)
    d = torch.from_numpy(data).cuda()
    sets = table1_settings() + table1_settings(extra_run_byte=True) + table1_settings(base=True)
    rows = sweep(d, sets)
    for s, r in zip(sets, rows):
        cuts = oracle.chunk(data, Params(*s))
        assert r["chunks"] == cuts.size
        assert r["mean_bytes"] == pytest.approx(data.size / cuts.size, abs=0.05)
        sizes = np.diff(np.concatenate([[0], cuts.astype(np.int64)]))
        assert r["at_max"] == pytest.approx(float((sizes == s[5]).mean()), abs=1e-4)


def test_target_limits_follow_sec_vi(seqcdc_lib):
    from paper_2505_21194_gb300.sweep import target_limits
    for kib in (4, 8, 16):
        o = oracle.presets(kib)
        assert target_limits(kib) == (o.min_size, o.max_size)


@pytest.mark.gpu
def test_search_means_equal_oracle(gpu):
    """Every mean the search reports (a wide tolerance keeps the whole small
    grid) equals the oracle's on the same sample, under both readings."""
    import torch
    from paper_2505_21194_gb300.sweep import search, target_limits
    data = W.uniform_random(4 << 20, 21)
    d = torch.from_numpy(data).cuda()
    res = search(d, targets_kib=(4, 16), seq_lengths=(4, 5), triggers=(50, 55),
                 skip_sizes=(256, 512), tol=10.0)
    checked = 0
    for kib, r in res.items():
        mn, mx = target_limits(kib)
        assert len(r["within"]) == 2 * 2 * 2 * 2        # the whole grid
        for row in r["within"]:
            q = Params(0, row["seq_length"] + row["reading"], row["skip_trigger"],
                       row["skip_size"], mn, mx)
            cuts = oracle.chunk(data, q)
            assert row["mean_bytes"] == pytest.approx(data.size / cuts.size, abs=0.05)
            checked += 1
        # Table I's row is in the grid: its means under both readings
        assert set(r["table1"]["mean_bytes_by_reading"]) == {0, 1}
    assert checked == 32
