"""Fingerprints and deduplication savings of a chunked input -- test
infrastructure only, like the rest of ``oracle/``.

The fingerprint of a chunk is its SHA-256 digest (the hash named for
fingerprinting in Sec. II), computed with the Python standard library's
hashlib; a chunk is stored once per distinct digest, and the savings are
1 - (bytes of distinct chunks) / (all bytes) (Eq. 1).  Pinned in
tests/test_fingerprint.py by the published SHA-256 known answers (the worked
examples of FIPS 180-2 Appendix B and the zero-length validation vector,
stored in tests/golden/sha256_known_answers.json) and by inputs whose distinct
chunks and savings are known by construction.
"""
from __future__ import annotations

import hashlib
from typing import Iterable, List, Tuple

import numpy as np


def chunk_ranges(offsets, cuts, cut_offsets) -> List[Tuple[int, int]]:
    """Absolute [a, b) of every chunk of a CSR batch of cut lists."""
    out = []
    offsets = np.asarray(offsets, dtype=np.int64)
    cuts = np.asarray(cuts, dtype=np.int64)
    co = np.asarray(cut_offsets, dtype=np.int64)
    for f in range(offsets.size - 1):
        prev = 0
        for c in cuts[co[f]:co[f + 1]].tolist():
            out.append((int(offsets[f]) + prev, int(offsets[f]) + c))
            prev = c
    return out


def fingerprints(data: np.ndarray, ranges: Iterable[Tuple[int, int]]) -> List[bytes]:
    mv = memoryview(np.ascontiguousarray(data))
    return [hashlib.sha256(mv[a:b]).digest() for a, b in ranges]


def distinct(ranges, digests) -> Tuple[int, int]:
    """(distinct chunks, their bytes): the first chunk with a digest counts."""
    seen, nbytes = set(), 0
    for (a, b), d in zip(ranges, digests):
        if d not in seen:
            seen.add(d)
            nbytes += b - a
    return len(seen), nbytes


def savings(total_bytes: int, distinct_bytes: int) -> float:
    return 1.0 - distinct_bytes / total_bytes if total_bytes else 0.0
