"""Fingerprints (SHA-256 of each chunk) and distinct-chunk counting.

Reference: the standard library's SHA-256 (hashlib) and ``oracle/dedup.py``,
pinned by the published known answers of the Secure Hash Standard
(``tests/golden/sha256_known_answers.json``: FIPS 180-2 Appendix B and the
zero-length SHAVS vector).  The GPU kernel is checked against the same known
answers, on message lengths around the padding boundaries (55/56/63/64/119/120
bytes), on chunks at every byte alignment, on the chunk lists the chunker
produces, and on inputs whose distinct-chunk count is known by construction.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import pytest

import oracle
from oracle import dedup as D
from paper_2505_21194_gb300 import workloads as W


_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sha256_known_answers.json")


def _known_answers():
    with open(_GOLDEN) as f:
        vecs = json.load(f)["vectors"]
    return [(v["name"], np.frombuffer((v["ascii"] * v["repeat"]).encode(), dtype=np.uint8),
             bytes.fromhex(v["sha256"])) for v in vecs]


def test_oracle_fingerprints_match_published_known_answers():
    """FIPS 180-2 Appendix B and the zero-length vector, through the oracle's
    fingerprint function (one chunk per message)."""
    for name, msg, digest in _known_answers():
        assert D.fingerprints(msg, [(0, msg.size)]) == [digest], name
    # the same messages side by side in one buffer, as chunks of a stream
    kas = _known_answers()
    data = np.concatenate([m for _, m, _ in kas])
    ends = np.cumsum([m.size for _, m, _ in kas])
    ranges = list(zip([0] + ends[:-1].tolist(), ends.tolist()))
    assert D.fingerprints(data, ranges) == [d for _, _, d in kas]


def test_oracle_distinct_and_savings_known_by_construction():
    x = W.uniform_random(5000, 1)
    y = W.uniform_random(3000, 2)
    data = np.concatenate([x, x, y, x])
    ranges = [(0, 5000), (5000, 10000), (10000, 13000), (13000, 18000)]
    n, b = D.distinct(ranges, D.fingerprints(data, ranges))
    assert (n, b) == (2, 8000)
    assert D.savings(18000, b) == pytest.approx(1 - 8000 / 18000)
    assert D.savings(0, 0) == 0.0
    # CSR ranges: file-relative cut lists, an empty file in the middle
    r = D.chunk_ranges([0, 10, 10, 25], [4, 10, 7, 15], [0, 2, 2, 4])
    assert r == [(0, 4), (4, 10), (10, 17), (17, 25)]


def test_oracle_digest_is_sha256_of_the_bytes():
    data = np.frombuffer(b"abc" + bytes(range(256)), dtype=np.uint8)
    d = D.fingerprints(data, [(0, 3), (3, 259), (0, 0)])
    assert d[0] == hashlib.sha256(b"abc").digest()
    assert d[1] == hashlib.sha256(bytes(range(256))).digest()
    assert d[2] == hashlib.sha256(b"").digest()


def test_abi_dedup_table_and_argument_checks(seqcdc_lib):
    s = seqcdc_lib
    assert s.seqcdc_dedup_table_bytes(0) == 4096
    assert s.seqcdc_dedup_table_bytes(1000) == 4 * 2048
    assert s.seqcdc_dedup_table_bytes(3000) == 4 * 8192
    lib = s.load_library()
    # nothing to do: no device call is made
    assert lib.seqcdc_fingerprint_batch(None, 0, None, 0, None, None, 0, None, None, None) == 0
    assert lib.seqcdc_fingerprint_batch(None, 0, None, 1, None, None, 5, None, None, None) == s.SEQCDC_EINVAL
    assert lib.seqcdc_dedup(None, None, 0, None, 0, None, None) == s.SEQCDC_EINVAL


def _gpu_digests(s, data, offs, cuts, co):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(data)).cuda()
    o = torch.from_numpy(np.asarray(offs, dtype=np.int64)).cuda()
    c = torch.from_numpy(np.asarray(cuts, dtype=np.int64)).cuda()
    cc = torch.from_numpy(np.asarray(co, dtype=np.int64)).cuda()
    r = s.BatchResult(c, cc)
    dig, sizes = s.fingerprint(d, o, r)
    return dig.cpu().numpy(), sizes.cpu().numpy(), (dig, sizes)


@pytest.mark.gpu
def test_gpu_sha256_lengths_and_alignments(gpu):
    s = gpu
    rng = np.random.default_rng(7)
    lengths = [0, 1, 3, 55, 56, 57, 63, 64, 65, 119, 120, 127, 128, 1000, 4096, 70001]
    # one file per (length, alignment): files packed back to back, so starts
    # fall on every byte offset
    files = []
    for L in lengths:
        for shift in range(4):
            files.append(rng.integers(0, 256, L + shift, dtype=np.uint8))
    sizes = np.array([f.size for f in files], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    data = np.concatenate(files)
    # each file: one chunk of the whole file, except a split after `shift`
    # bytes when that leaves two non-empty chunks
    cuts, co = [], [0]
    for k, f in enumerate(files):
        shift = k % 4
        if 0 < shift < f.size:
            cuts += [shift, f.size]
        elif f.size:
            cuts += [f.size]
        co.append(len(cuts))
    got, gsz, _ = _gpu_digests(s, data, offs, cuts, co)
    ranges = D.chunk_ranges(offs, cuts, co)
    exp = D.fingerprints(data, ranges)
    assert got.shape == (len(ranges), 32)
    for i, (a, b) in enumerate(ranges):
        assert got[i].tobytes() == exp[i], (i, a, b)
        assert gsz[i] == b - a


@pytest.mark.gpu
def test_gpu_fingerprints_of_chunker_output_and_dedup(gpu):
    import torch
    s = gpu
    base, _ = W.file_batch(30, seed=5)
    # repeat the batch's bytes so that whole files recur
    data = np.concatenate([base, base[: base.size // 2], base])
    nf = 60
    offs = np.linspace(0, data.size, nf + 1).astype(np.int64)
    p = s.seqcdc_params(8, 0)
    d = torch.from_numpy(data).cuda()
    o = torch.from_numpy(offs).cuda()
    r = s.chunk_batch(d, o, p)
    dig, sizes = s.fingerprint(d, o, r)
    ranges = D.chunk_ranges(offs, r.cuts.cpu().numpy(), r.cut_offsets.cpu().numpy())
    exp = D.fingerprints(data, ranges)
    got = dig.cpu().numpy()
    assert all(got[i].tobytes() == exp[i] for i in range(len(ranges)))
    assert (sizes.cpu().numpy() == np.array([b - a for a, b in ranges])).all()
    n, nbytes = s.dedup(dig, sizes)
    assert (n, nbytes) == D.distinct(ranges, exp)
    assert 0 < nbytes < data.size
    # all chunks distinct; no chunks
    n2, b2 = s.dedup(dig[:1], sizes[:1])
    assert (n2, b2) == (1, int(sizes[0]))
    assert s.dedup(dig[:0], sizes[:0]) == (0, 0)


@pytest.mark.gpu
def test_gpu_sha256_published_known_answers(gpu):
    """The GPU kernel on FIPS 180-2 Appendix B's three messages, each a chunk
    of its own file and, shifted to every alignment, a chunk inside a file
    (the zero-length message cannot be a chunk: chunks are never empty)."""
    s = gpu
    kas = [k for k in _known_answers() if k[1].size > 0]
    files, cuts, co, expect = [], [], [0], []
    for name, msg, digest in kas:
        for shift in range(4):
            pad = np.full(shift, 0x5A, dtype=np.uint8)
            files.append(np.concatenate([pad, msg]))
            if shift:
                cuts += [shift, shift + msg.size]
                expect += [None, (name, digest)]
            else:
                cuts += [msg.size]
                expect += [(name, digest)]
            co.append(len(cuts))
    offs = np.concatenate([[0], np.cumsum([f.size for f in files])])
    got, gsz, _ = _gpu_digests(s, np.concatenate(files), offs, cuts, co)
    for i, e in enumerate(expect):
        if e is not None:
            assert got[i].tobytes() == e[1], (e[0], i)
