"""One 64 GiB stream of adversarial 16 MiB blocks, 16 KB setting.

The stream cycles uniform random -> zeros -> ramp 0..255 -> saw-tooth (period
3..9 drawn per block); every block is a function of (seed, index), so the host
regenerates any part of it without holding 64 GiB.  Zeros give no run ends
(forced cuts at max_size), ramps and long saw-tooth periods give a run end at
every byte (more natural cuts per segment than a segment tabulates, so those
segments go through the exact repair pass), and short periods give neither
order of pair in long stretches.

The GPU chunks the whole stream in one call.  Checked against the oracle:
  - every cut of the first 1 GiB, with the streaming oracle;
  - 200 cuts drawn at random over the whole stream, each recomputed by the
    oracle from the cut before it (a chunk depends only on the bytes from its
    start to start + max_size, so this is the exact rule, cut by cut);
  - at every cut, the size bounds of Sec. VI (all chunks but the last within
    [min, max]) and the stream end as the last cut.
"""
from __future__ import annotations

import functools

import numpy as np
import pytest

import oracle
from paper_2505_21194_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

BLOCK = 16 << 20
NBLOCKS = 4096          # 64 GiB
SEED = 0


@functools.lru_cache(maxsize=8)
def _block(i: int) -> np.ndarray:
    return W.adversarial_block(i, SEED, BLOCK)


def _bytes(lo: int, hi: int) -> np.ndarray:
    """Stream bytes [lo, hi) from the generator."""
    out = []
    pos = lo
    while pos < hi:
        b, off = divmod(pos, BLOCK)
        take = min(hi - pos, BLOCK - off)
        out.append(_block(b)[off:off + take])
        pos += take
    return np.concatenate(out) if out else np.empty(0, np.uint8)


def test_config5_adversarial_64gib(gpu):
    import torch
    s = gpu
    p = s.seqcdc_params(16, 0)
    n = NBLOCKS * BLOCK
    need = n + s.seqcdc_workspace_size(p, n, 1) + (n // p.min_size + 2) * 8
    free, _ = torch.cuda.mem_get_info()
    if free < need + (4 << 30):
        pytest.skip("needs %.1f GiB of device memory" % (need / 2**30))
    d = torch.empty(n, dtype=torch.uint8, device="cuda")
    for i in range(NBLOCKS):
        d[i * BLOCK:(i + 1) * BLOCK].copy_(torch.from_numpy(W.adversarial_block(i, SEED, BLOCK)))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    cuts_d = s.chunk(d, p)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    print("config 5: %d cuts in %.1f ms (%.1f GB/s)" % (cuts_d.numel(), ms, n / ms / 1e6))
    cuts = cuts_d.cpu().numpy().astype(np.uint64)
    del d, cuts_d
    torch.cuda.empty_cache()

    # Sizes (Sec. VI) and the stream end.
    assert int(cuts[-1]) == n
    gaps = np.diff(np.concatenate([[0], cuts.astype(np.int64)]))
    assert (gaps[:-1] >= p.min_size).all() and (gaps <= p.max_size).all()

    op = oracle.Params(p.mode, p.seq_length, p.skip_trigger, p.skip_size,
                       p.min_size, p.max_size)
    # The first 1 GiB, exactly.
    head = 64 * BLOCK
    exp = np.concatenate(list(oracle.chunk_stream((_block(i) for i in range(64)), op)))
    exp = exp[exp < head]
    got = cuts[cuts < head]
    assert got.size == exp.size and np.array_equal(got, exp)

    # Sampled cuts over the whole stream, each from the one before it.
    rng = np.random.default_rng(5)
    for k in sorted(rng.choice(cuts.size, 200, replace=False).tolist()):
        start = int(cuts[k - 1]) if k else 0
        window = _bytes(start, min(start + p.max_size, n))
        first = int(oracle.chunk(window, op)[0])
        assert start + first == int(cuts[k]), (k, start)
