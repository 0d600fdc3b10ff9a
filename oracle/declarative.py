"""Second, independently written SeqCDC formulation -- TEST INFRASTRUCTURE ONLY.

Where ``seqcdc_oracle.c`` walks the bytes one pair at a time with two counters,
this module restates the same rules (Sec. III.A-C and the maximum chunk size
of Sec. IV) from whole-input prefix quantities and searches:

* ``run[j]``  -- number of consecutive target-order pairs ending with the pair
  (b[j-1], b[j]);
* ``opp[j]``  -- cumulative count of opposing-order pairs among the pairs
  (b[0], b[1]) .. (b[j-1], b[j]).

A scan region that starts at byte ``i`` (the first byte after the sub-minimum
region, Sec. III.B, or after a skipped region, Sec. III.C) then has

* its first boundary at the smallest ``e >= i + SeqLength - 1`` with
  ``run[e] >= SeqLength - 1`` (the pairs of the run all lie after ``i``), the
  cut falling right after byte ``e``;
* its skip at the smallest ``s >= i + 1`` with
  ``opp[s] - opp[i] == SkipTrigger``, after which the next region starts at
  ``s + 1 + SkipSize``;

and the earlier of the two inside the chunk's size limit decides.  It is pure
Python and meant for inputs of at most a few thousand bytes.
"""
from __future__ import annotations

from bisect import bisect_left


def _target(mode: int, prev: int, cur: int) -> bool:
    return cur > prev if mode == 0 else cur < prev


def _opposing(mode: int, prev: int, cur: int) -> bool:
    return cur < prev if mode == 0 else cur > prev


def chunk(data, p) -> list[int]:
    """Chunk end offsets of ``data`` under parameters ``p`` (oracle.Params)."""
    b = list(bytes(data)) if not isinstance(data, list) else data
    n = len(b)
    R, T, S = p.seq_length, p.skip_trigger, p.skip_size
    mn, mx = p.min_size, p.max_size

    run = [0] * n
    opp = [0] * n
    for j in range(1, n):
        run[j] = run[j - 1] + 1 if _target(p.mode, b[j - 1], b[j]) else 0
        opp[j] = opp[j - 1] + (1 if _opposing(p.mode, b[j - 1], b[j]) else 0)
    # Positions where a run of SeqLength bytes ends (sorted).
    ends = [j for j in range(n) if run[j] >= R - 1]

    cuts = []
    c = 0
    while c < n:
        limit = min(c + mx, n)
        i = c + max(mn - R, 0)
        cut = limit
        while i + 1 < limit:
            k = bisect_left(ends, i + R - 1)
            e = ends[k] if k < len(ends) and ends[k] < limit else None
            s = None
            if T > 0:
                s_idx = bisect_left(opp, opp[i] + T, lo=i + 1, hi=limit)
                if s_idx < limit:
                    s = s_idx
            if e is not None and (s is None or e < s):
                cut = e + 1
                break
            if s is None:
                break
            i = s + 1 + S
        cuts.append(cut)
        c = cut
    return cuts
