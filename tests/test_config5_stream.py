"""One 64 GiB stream of adversarial 16 MiB blocks, 16 KB setting.

The stream cycles uniform random -> zeros -> ramp 0..255 -> saw-tooth (period
3..9 drawn per block); every block is a function of (seed, index), so the host
produces the stream block by block without holding 64 GiB.  Zeros give no run
ends (forced cuts at max_size), ramps and long saw-tooth periods give a run
end at every byte (more natural cuts per segment than a segment tabulates, so
those segments go through the exact repair pass), and short periods give
neither order of pair in long stretches.

Each block is generated once: it is copied to the device and handed to the
streaming oracle (the sequential chunker of Sec. III.A-C and Sec. IV, resumed
at its last proven cut from block to block), so the oracle sees exactly the
bytes the GPU chunks.  The GPU then chunks the whole stream in one call, and
its cut list must equal the oracle's over the FULL stream, cut for cut; the
size bounds of Sec. VI are checked as well.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from paper_2505_21194_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

BLOCK = 16 << 20
NBLOCKS = 4096          # 64 GiB
SEED = 0


def _run(s, p, nblocks, tuning=None):
    """Upload the first ``nblocks`` blocks, chunk them on the device in one
    call; returns (GPU cuts, oracle cuts, ms)."""
    import torch
    n = nblocks * BLOCK
    op = oracle.Params(p.mode, p.seq_length, p.skip_trigger, p.skip_size,
                       p.min_size, p.max_size)
    d = torch.empty(n, dtype=torch.uint8, device="cuda")

    def blocks():
        for i in range(nblocks):
            b = W.adversarial_block(i, SEED, BLOCK)
            d[i * BLOCK:(i + 1) * BLOCK].copy_(torch.from_numpy(b))
            yield b

    t = time.perf_counter()
    exp = np.concatenate(list(oracle.chunk_stream(blocks(), op)))
    print("config 5: oracle over %d bytes in %.1f s (with generation and upload)"
          % (n, time.perf_counter() - t))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    cuts_d = s.chunk(d, p, tuning)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    got = cuts_d.cpu().numpy().astype(np.uint64)
    del d, cuts_d
    torch.cuda.empty_cache()
    return got, exp, ms


def test_config5_adversarial_64gib_full_stream(gpu):
    import torch
    s = gpu
    p = s.seqcdc_params(16, 0)
    n = NBLOCKS * BLOCK
    need = n + s.seqcdc_workspace_size(p, n, 1) + (n // p.min_size + 2) * 8
    free, _ = torch.cuda.mem_get_info()
    if free < need + (4 << 30):
        pytest.skip("needs %.1f GiB of device memory" % (need / 2**30))
    got, exp, ms = _run(s, p, NBLOCKS)
    print("config 5: %d cuts in %.1f ms (%.1f GB/s)" % (got.size, ms, n / ms / 1e6))

    # Sizes (Sec. VI) and the stream end.
    assert int(got[-1]) == n
    gaps = np.diff(np.concatenate([[0], got.astype(np.int64)]))
    assert (gaps[:-1] >= p.min_size).all() and (gaps <= p.max_size).all()
    # Every cut of the stream, against the oracle.
    assert exp.size == got.size, (exp.size, got.size)
    bad = np.nonzero(exp != got)[0]
    assert bad.size == 0, "first difference at cut %d: %d vs oracle %d" % (
        bad[0], got[bad[0]], exp[bad[0]])
