"""Parameter sweep on the GPU: mean chunk size over (SeqLength, SkipTrigger,
SkipSize), the BASE variant (no skipping) included.

Sec. IV sets SeqLength, SkipTrigger and SkipSize so that the mean chunk size
meets a target (Table I), and Sec. VI uses min = 1/2 and max = 2 times the
target.  The sweep chunks a device-resident sample at each setting and
reports the mean and the fraction of chunks cut at max_size.  Chunking the
same sample with seq_length = SeqLength and SeqLength + 1 shows which count of
the run length (bytes or comparisons) gives Table I's targets on that data.
"""
from __future__ import annotations

from typing import Dict, Iterable, List, Optional, Tuple

import numpy as np

from . import seqcdc


def mean_chunk(d_data, p, tuning=None) -> Tuple[float, float, int]:
    """(mean chunk bytes, fraction of chunks at max_size, chunks) of one
    device-resident stream."""
    cuts = seqcdc.chunk(d_data, p, tuning)
    n = cuts.numel()
    if n == 0:
        return 0.0, 0.0, 0
    sizes = cuts.diff(prepend=cuts.new_zeros(1))
    at_max = float((sizes == p.max_size).float().mean().item())
    return d_data.numel() / n, at_max, n


def sweep(d_data, settings: Iterable[Tuple[int, int, int, int, int, int]],
          tuning=None) -> List[Dict]:
    """settings: (mode, seq_length, skip_trigger, skip_size, min, max)."""
    out = []
    for mode, R, T, S, mn, mx in settings:
        p = seqcdc.Params(mode, R, T, S, mn, mx)
        mean, at_max, n = mean_chunk(d_data, p, tuning)
        out.append({"mode": mode, "seq_length": R, "skip_trigger": T, "skip_size": S,
                    "min": mn, "max": mx, "chunks": n, "mean_bytes": round(mean, 1),
                    "at_max": round(at_max, 4)})
    return out


def table1_settings(extra_run_byte: bool = False, base: bool = False):
    """Table I's three settings (4/8/16 KB, increasing mode); optionally with
    one more byte per run (the other reading of SeqLength) or without skipping
    (the BASE variant)."""
    out = []
    for kib in (4, 8, 16):
        p = seqcdc.seqcdc_params(kib, 0)
        out.append((0, p.seq_length + (1 if extra_run_byte else 0),
                    0 if base else p.skip_trigger, p.skip_size, p.min_size, p.max_size))
    return out
