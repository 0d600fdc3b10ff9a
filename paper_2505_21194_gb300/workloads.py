"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no chunking arithmetic: it only produces byte streams and
CSR file batches with the shapes and content mixes of the benchmark workloads
(uniform random bytes, order-1 Markov text, backup-like versioned streams,
log-normal file batches, adversarial block cycles).  Every generator draws
from numpy's PCG64 (``numpy.random.default_rng``), which gives the same bytes
on every platform for the same seed.
"""
from __future__ import annotations

import numpy as np

MIB = 1 << 20
KIB = 1 << 10

# Printable ASCII 0x20..0x7E plus newline: the 96 text symbols.
TEXT_SYMBOLS = np.array(list(range(0x20, 0x7F)) + [0x0A], dtype=np.uint8)


def uniform_random(n: int, seed: int) -> np.ndarray:
    """``n`` uniform random bytes."""
    rng = np.random.default_rng(seed)
    return np.frombuffer(rng.bytes(n), dtype=np.uint8).copy()


def _markov_tables(rng, fanout: int = 12, skew: float = 1.2):
    """Sparse, skewed order-1 transition tables over the 96 text symbols."""
    nsym = TEXT_SYMBOLS.size
    succ = np.empty((nsym, fanout), dtype=np.int64)
    for s in range(nsym):
        succ[s] = rng.permutation(nsym)[:fanout]
    w = 1.0 / np.arange(1, fanout + 1) ** skew
    cdf = np.cumsum(w) / w.sum()
    cdf[-1] = 1.0
    return succ, cdf


def markov_text(n: int, seed: int, chain_len: int = 4096) -> np.ndarray:
    """``n`` bytes of order-1 Markov text over 96 printable symbols.

    The stream is cut into independent chains of ``chain_len`` symbols that
    are advanced in lockstep (each chain starts from a random symbol), so the
    generator runs at numpy speed; within a chain every symbol depends on the
    previous one through a sparse, skewed transition table.
    """
    rng = np.random.default_rng(seed)
    succ, cdf = _markov_tables(rng)
    nchains = max(1, -(-n // chain_len))
    out = np.empty((nchains, chain_len), dtype=np.int64)
    state = rng.integers(0, TEXT_SYMBOLS.size, nchains)
    u = rng.random((chain_len, nchains))
    for k in range(chain_len):
        out[:, k] = state
        pick = np.searchsorted(cdf, u[k], side="right")
        np.minimum(pick, cdf.size - 1, out=pick)
        state = succ[state, pick]
    return TEXT_SYMBOLS[out.reshape(-1)[:n]]


def mixed_base(n: int, seed: int, block: int = 64 * KIB) -> np.ndarray:
    """Blocks of ``block`` bytes, exactly half uniform random and half text.

    Which blocks are text is a seeded permutation.
    """
    rng = np.random.default_rng(seed)
    nblk = -(-n // block)
    is_text = np.zeros(nblk, dtype=bool)
    is_text[rng.permutation(nblk)[: nblk // 2]] = True
    rnd = uniform_random(nblk * block, int(rng.integers(1 << 62)))
    txt = markov_text(int(is_text.sum()) * block, int(rng.integers(1 << 62)))
    out = rnd.reshape(nblk, block)
    out[is_text] = txt.reshape(-1, block)
    return out.reshape(-1)[:n].copy()


def apply_edits(prev: np.ndarray, rng, mean_edits: float = 200.0,
                min_len: int = 1 * KIB, max_len: int = 4 * KIB) -> np.ndarray:
    """One new version: Poisson(mean_edits) edits of min_len..max_len bytes.

    Edit positions are uniform over ``prev`` and applied left to right in one
    pass; insert, delete and overwrite are equally likely; inserted and
    overwriting bytes are uniform random.  An edit that starts inside a range
    an earlier edit of the same version consumed starts at that range's end.
    """
    k = int(rng.poisson(mean_edits))
    pos = np.sort(rng.integers(0, max(prev.size, 1), k))
    lens = rng.integers(min_len, max_len + 1, k)
    kinds = rng.integers(0, 3, k)  # 0 insert, 1 delete, 2 overwrite
    pieces = []
    cur = 0
    for p0, ln, kd in zip(pos.tolist(), lens.tolist(), kinds.tolist()):
        p0 = max(p0, cur)
        if p0 > prev.size:
            break
        pieces.append(prev[cur:p0])
        if kd == 0:
            pieces.append(np.frombuffer(rng.bytes(ln), dtype=np.uint8))
            cur = p0
        elif kd == 1:
            cur = min(prev.size, p0 + ln)
        else:
            end = min(prev.size, p0 + ln)
            pieces.append(np.frombuffer(rng.bytes(end - p0), dtype=np.uint8))
            cur = end
    pieces.append(prev[cur:])
    return np.concatenate(pieces)


def backup_stream(seed: int = 0, base_size: int = 16 * MIB,
                  versions: int = 64):
    """Backup-like stream: ``versions`` successive edited copies of a base.

    Version 0 is a ``mixed_base`` of ``base_size`` bytes; version k applies
    ``apply_edits`` to version k-1.  Returns (stream, version_offsets) with the
    versions concatenated back to back.
    """
    rng = np.random.default_rng(seed)
    v = mixed_base(base_size, int(rng.integers(1 << 62)))
    parts = [v]
    for _ in range(versions - 1):
        v = apply_edits(v, rng)
        parts.append(v)
    offs = np.zeros(versions + 1, dtype=np.uint64)
    np.cumsum([x.size for x in parts], out=offs[1:])
    return np.concatenate(parts), offs


def lognormal_sizes(nfiles: int, seed: int, median: int = 256 * KIB,
                    sigma: float = 1.5, lo: int = 4 * KIB,
                    hi: int = 64 * MIB) -> np.ndarray:
    """File sizes: log-normal (median, sigma), floored, clamped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    s = np.floor(median * np.exp(sigma * rng.standard_normal(nfiles)))
    return np.clip(s, lo, hi).astype(np.int64)


def file_batch(nfiles: int, seed: int, median: int = 256 * KIB,
               sigma: float = 1.5, lo: int = 4 * KIB, hi: int = 64 * MIB,
               block: int = 64 * KIB, text_pool: int = 64 * MIB):
    """CSR batch of files with log-normal sizes and half random / half text.

    Each file is a sequence of ``block``-byte pieces; a seeded coin picks
    random bytes or a slice (at a random offset) of a seeded Markov-text pool.
    Returns (data, offsets) with ``offsets`` of length nfiles+1 (uint64).
    """
    rng = np.random.default_rng(seed)
    sizes = lognormal_sizes(nfiles, int(rng.integers(1 << 62)), median, sigma,
                            lo, hi)
    offs = np.zeros(nfiles + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offs[1:])
    total = int(offs[-1])
    data = uniform_random(total, int(rng.integers(1 << 62)))
    pool = markov_text(min(text_pool, max(total, block)),
                       int(rng.integers(1 << 62)))
    nblk = -(-total // block)
    text_blocks = np.nonzero(rng.random(nblk) < 0.5)[0]
    starts = rng.integers(0, pool.size - block + 1, text_blocks.size)
    for bi, st in zip(text_blocks.tolist(), starts.tolist()):
        a = bi * block
        ln = min(block, total - a)
        data[a:a + ln] = pool[st:st + ln]
    return data, offs


ADVERSARIAL_KINDS = ("random", "zeros", "ramp", "sawtooth")


def adversarial_block(index: int, seed: int, block: int = 16 * MIB) -> np.ndarray:
    """Block ``index`` of the adversarial stream.

    Blocks cycle uniform random -> zeros -> ramp 0..255 -> saw-tooth; the
    saw-tooth period is drawn from 3..9 per block and its values step by
    256 // period from 0.  Each block depends only on (seed, index), so the
    stream can be produced block by block.
    """
    kind = ADVERSARIAL_KINDS[index % 4]
    if kind == "random":
        return uniform_random(block, (seed << 32) ^ index)
    if kind == "zeros":
        return np.zeros(block, dtype=np.uint8)
    if kind == "ramp":
        return _tile(np.arange(256, dtype=np.uint8), block)
    rng = np.random.default_rng((seed << 32) ^ index)
    period = int(rng.integers(3, 10))
    return _tile((np.arange(period) * (256 // period)).astype(np.uint8), block)


def _tile(pattern: np.ndarray, n: int) -> np.ndarray:
    """``pattern`` repeated from its start, cut to ``n`` bytes."""
    reps = -(-n // pattern.size)
    return np.tile(pattern, reps)[:n].copy()


def adversarial_stream(nblocks: int, seed: int = 0, block: int = 16 * MIB):
    """Iterator over the blocks of an adversarial stream of nblocks blocks."""
    for i in range(nblocks):
        yield adversarial_block(i, seed, block)
