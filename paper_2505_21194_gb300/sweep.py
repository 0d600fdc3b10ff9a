"""Parameter sweep and search on the GPU: mean chunk size over (SeqLength,
SkipTrigger, SkipSize), the BASE variant (no skipping) included, and the
Monte-Carlo search of Sec. V over a grid of them for the 4 / 8 / 16 KiB
targets (``search``).

Sec. IV sets SeqLength, SkipTrigger and SkipSize so that the mean chunk size
meets a target (Table I), and Sec. VI uses min = 1/2 and max = 2 times the
target.  The sweep chunks a device-resident sample at each setting and
reports the mean and the fraction of chunks cut at max_size.  Chunking the
same sample with seq_length = SeqLength and SeqLength + 1 shows which count of
the run length (bytes or comparisons) gives Table I's targets on that data.
"""
from __future__ import annotations

from typing import Dict, Iterable, List, Tuple

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


def target_limits(kib: int) -> Tuple[int, int]:
    """Sec. VI's minimum and maximum chunk sizes for an expected size of
    `kib` KiB: half and twice the expected size, with a 1 KiB minimum for
    the 4 KiB setting."""
    return (1024 if kib == 4 else kib * 512), kib * 2048


def search(d_data, targets_kib=(4, 8, 16), seq_lengths=range(3, 9),
           triggers=range(20, 81, 5), skip_sizes=(128, 256, 512),
           readings=(0, 1), mode: int = 0, tol: float = 0.05) -> Dict:
    """Monte-Carlo search of Sec. V ("Obtaining parameter values"): the mean
    chunk size of every (SeqLength, SkipTrigger, SkipSize) on a
    device-resident sample, for each target with Sec. VI's min / max, under
    each reading of SeqLength (0: a run of SeqLength bytes, the reading this
    library takes; 1: SeqLength comparisons, one more byte).  Returns, per
    target, every setting whose mean lies within `tol` of the target and the
    means of Table I's row under both readings."""
    import torch
    n = int(d_data.numel())
    dev = d_data.device
    cap = n // 1024 + 1
    cuts = torch.empty(cap, dtype=torch.int64, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    ws_bytes = 0
    for kib in targets_kib:
        mn, mx = target_limits(kib)
        for rl in (min(seq_lengths), max(seq_lengths) + max(readings)):
            p = seqcdc.make_params(mode, rl, 50, 256, mn, mx)
            ws_bytes = max(ws_bytes, seqcdc.seqcdc_workspace_size(p, n, 1))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    table1 = {kib: seqcdc.seqcdc_params(kib, mode) for kib in targets_kib}
    out = {}
    for kib in targets_kib:
        mn, mx = target_limits(kib)
        target = kib * 1024
        rows, t1 = [], {}
        for reading in readings:
            for R in seq_lengths:
                for T in triggers:
                    for S in skip_sizes:
                        p = seqcdc.make_params(mode, R + reading, T, S, mn, mx)
                        seqcdc.seqcdc_chunk(p, d_data, n, cuts, cap, count, ws, ws_bytes)
                        st = seqcdc.seqcdc_status(ws)
                        if st != seqcdc.SEQCDC_OK:
                            raise seqcdc.SeqCDCError(st, "sweep.search (device)")
                        k = int(count.item())
                        mean = n / k if k else 0.0
                        row = {"seq_length": R, "skip_trigger": T, "skip_size": S,
                               "reading": reading, "mean_bytes": round(mean, 1)}
                        q = table1[kib]
                        if (R, T, S) == (q.seq_length, q.skip_trigger, q.skip_size):
                            t1[reading] = row["mean_bytes"]
                        if abs(mean - target) <= tol * target:
                            rows.append(row)
        q = table1[kib]
        out[kib] = {"target_bytes": target, "min": mn, "max": mx, "within": rows,
                    "table1": {"seq_length": q.seq_length, "skip_trigger": q.skip_trigger,
                               "skip_size": q.skip_size,
                               "mean_bytes_by_reading": t1,
                               "within_by_reading": {r: abs(m - target) <= tol * target
                                                     for r, m in t1.items()}}}
    return out
