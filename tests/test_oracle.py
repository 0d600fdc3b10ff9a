"""CPU pins of the oracle (no GPU): worked examples, closed forms, invariants,
brute force against an independently written formulation, and mutation
checks showing that plausible mistakes in the oracle fail these pins."""
from __future__ import annotations

import ctypes
import itertools
import json
import os
import random
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import Params, declarative

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        d = json.load(f)
    return Params(**d["params"]), np.array(d["bytes"], dtype=np.uint8), d["cuts"]


def _u8(seq):
    return np.array(seq, dtype=np.uint8)


# ---------------------------------------------------------------------------
# Worked examples.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["hand_example.json", "trigger_example.json",
                                  "vector_example.json"])
def test_worked_examples(name):
    p, b, cuts = _golden(name)
    assert oracle.chunk(b, p).tolist() == cuts
    assert declarative.chunk(b.tolist(), p) == cuts


def test_vector_example_boundary_offset():
    # Sec. III.D: first combined-mask bit at index 61, boundary SeqLength ahead.
    with open(os.path.join(GOLDEN, "vector_example.json")) as f:
        d = json.load(f)
    assert d["cuts"][0] == d["first_mask_bit"] + d["params"]["seq_length"]


def test_presets_table1():
    # Table I and Sec. VI min/max (1 KB minimum for 4 KB).
    assert oracle.presets(4) == Params(0, 5, 55, 256, 1024, 8192)
    assert oracle.presets(8) == Params(0, 5, 50, 256, 4096, 16384)
    assert oracle.presets(16, 1) == Params(1, 5, 50, 512, 8192, 32768)
    with pytest.raises(ValueError):
        oracle.presets(32)


# ---------------------------------------------------------------------------
# Closed forms.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kib", [4, 8, 16])
@pytest.mark.parametrize("mode", [0, 1])
def test_all_equal_bytes_cut_at_max(kib, mode):
    p = oracle.presets(kib, mode)
    n = 5 * p.max_size + 123
    cuts = oracle.chunk(np.full(n, 77, np.uint8), p).tolist()
    expect = list(range(p.max_size, n, p.max_size)) + [n]
    assert cuts == expect


def test_decreasing_mode_on_ramp_cuts_at_max():
    # A 0..255 ramp has no strictly decreasing pair except the wraps.
    p = oracle.presets(8, oracle.DECREASING)
    n = 3 * p.max_size + 7
    ramp = (np.arange(n) % 256).astype(np.uint8)
    assert oracle.chunk(ramp, p).tolist() == list(range(p.max_size, n, p.max_size)) + [n]


def _no_skip_closed_form(b, p):
    """With skipping off, a chunk from c ends at the first e in [c+min, limit]
    such that b[e-R .. e-1] is strictly monotone, else at the limit."""
    x = b.astype(np.int16)
    d = np.diff(x)
    t = (d > 0) if p.mode == 0 else (d < 0)       # t[k]: pair (k, k+1)
    R = p.seq_length
    # good[e]: bytes e-R .. e-1 strictly monotone (pairs e-R .. e-2)
    n = b.size
    good = np.zeros(n + 1, bool)
    if n >= R:
        w = np.lib.stride_tricks.sliding_window_view(t, R - 1).all(axis=1)
        good[R:] = w  # window starting at pair e-R -> e = start + R
    cuts, c = [], 0
    while c < n:
        limit = min(c + p.max_size, n)
        lo = c + max(p.min_size, R)
        cand = np.nonzero(good[lo:limit + 1])[0]
        cut = lo + int(cand[0]) if cand.size else limit
        cuts.append(cut)
        c = cut
    return cuts


@pytest.mark.parametrize("seed", range(6))
def test_no_skip_matches_closed_form(seed):
    rng = np.random.default_rng(seed)
    alphabet = [3, 16, 256][seed % 3]
    b = rng.integers(0, alphabet, 20000).astype(np.uint8)
    R = 3 + seed % 4
    p = Params(seed % 2, R, 0, 0, R + 5 * seed + 1, R + 5 * seed + 300)
    assert oracle.chunk(b, p).tolist() == _no_skip_closed_form(b, p)


# ---------------------------------------------------------------------------
# Invariants.
# ---------------------------------------------------------------------------
def _random_input(rng, n):
    kind = rng.integers(0, 3)
    if kind == 0:
        return rng.integers(0, 256, n).astype(np.uint8)
    if kind == 1:
        return rng.integers(0, 4, n).astype(np.uint8)
    return (np.cumsum(rng.integers(-3, 4, n)) % 256).astype(np.uint8)


@pytest.mark.parametrize("seed", range(8))
def test_tiling_and_sizes(seed):
    rng = np.random.default_rng(100 + seed)
    p = [oracle.presets(4), oracle.presets(8, 1), oracle.presets(16),
         Params(seed % 2, 4, 7, 33, 50, 400)][seed % 4]
    n = int(rng.integers(1, 300000))
    cuts = oracle.chunk(_random_input(rng, n), p)
    assert cuts[-1] == n
    sizes = np.diff(np.concatenate([[0], cuts.astype(np.int64)]))
    assert (sizes > 0).all()
    assert (sizes[:-1] >= p.min_size).all() and (sizes <= p.max_size).all()


@pytest.mark.parametrize("seed", range(6))
def test_prefix_property(seed):
    # A cut e depends only on bytes before e.
    rng = np.random.default_rng(200 + seed)
    p = [oracle.presets(8), Params(1, 3, 5, 17, 20, 300)][seed % 2]
    b = _random_input(rng, 60000)
    full = oracle.chunk(b, p).tolist()
    for m in rng.integers(1, b.size, 5).tolist():
        part = oracle.chunk(b[:m], p).tolist()
        assert part == [c for c in full if c < m] + [m]


@pytest.mark.parametrize("seed", range(4))
def test_concatenation_at_a_cut(seed):
    rng = np.random.default_rng(300 + seed)
    p = oracle.presets([4, 8, 16, 8][seed], seed % 2)
    b = _random_input(rng, 200000)
    full = oracle.chunk(b, p).tolist()
    a = full[len(full) // 3]
    tail = (oracle.chunk(b[a:], p) + a).tolist()
    assert full == [c for c in full if c <= a] + tail


@pytest.mark.parametrize("seed", range(4))
def test_mode_duality(seed):
    rng = np.random.default_rng(400 + seed)
    b = _random_input(rng, 100000)
    for kib in (4, 8, 16):
        inc = oracle.chunk(255 - b, oracle.presets(kib, 0)).tolist()
        dec = oracle.chunk(b, oracle.presets(kib, 1)).tolist()
        assert inc == dec


def test_edit_locality():
    # Cuts at or before an edit position do not move (Sec. IV), and the chain
    # re-synchronises after the edit.
    rng = np.random.default_rng(7)
    p = oracle.presets(8)
    b = rng.integers(0, 256, 4 << 20).astype(np.uint8)
    full = oracle.chunk(b, p)
    pos = 1 << 20
    edited = np.concatenate([b[:pos], rng.integers(0, 256, 3000).astype(np.uint8),
                             b[pos:]])
    cuts2 = oracle.chunk(edited, p)
    before = full[full <= pos]
    assert cuts2[: before.size].tolist() == before.tolist()
    shifted = set((full[full > pos + 3000] + 3000).tolist())
    assert len(shifted & set(cuts2.tolist())) > 0.9 * len(shifted)


def test_empty_and_tiny_inputs():
    p = oracle.presets(8)
    assert oracle.chunk(np.empty(0, np.uint8), p).tolist() == []
    assert oracle.chunk(_u8([5]), p).tolist() == [1]
    assert oracle.chunk(_u8([1, 2, 3, 4, 5, 6]), p).tolist() == [6]


def test_mean_chunk_size_on_random_data():
    # Soft check of Sec. V (parameters chosen by simulation on random data):
    # chunks spread between min and max, none below min except the tail.
    b = np.random.default_rng(11).integers(0, 256, 32 << 20).astype(np.uint8)
    for kib in (4, 8, 16):
        p = oracle.presets(kib)
        cuts = oracle.chunk(b, p)
        mean = b.size / cuts.size
        assert p.min_size < mean < p.max_size


def test_batch_and_stream_agree_with_single():
    rng = np.random.default_rng(5)
    p = oracle.presets(4)
    sizes = rng.integers(0, 50000, 40)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    data = rng.integers(0, 256, int(offs[-1])).astype(np.uint8)
    cuts, co = oracle.chunk_batch(data, offs, p)
    cuts_t, co_t = oracle.chunk_batch_threaded(data, offs, p, 4)
    assert cuts.tolist() == cuts_t.tolist() and co.tolist() == co_t.tolist()
    for f in range(40):
        one = oracle.chunk(data[offs[f]:offs[f + 1]], p)
        assert cuts[co[f]:co[f + 1]].tolist() == one.tolist()
    blocks = np.array_split(data, 7)
    streamed = np.concatenate(list(oracle.chunk_stream(blocks, p)))
    assert streamed.tolist() == oracle.chunk(data, p).tolist()


# ---------------------------------------------------------------------------
# Brute force against the declarative formulation.
# ---------------------------------------------------------------------------
def _grid():
    for mode in (0, 1):
        for R in (2, 3):
            for T in (0, 1, 2, 3):
                for S in (0, 2):
                    for mn, mx in ((1, 3), (2, 5), (3, 3), (4, 9)):
                        yield Params(mode, R, T, S, mn, mx)


def test_exhaustive_small_alphabet():
    params = list(_grid())
    strings = [list(s) for L in range(0, 7)
               for s in itertools.product(range(4), repeat=L)]
    offs = np.concatenate([[0], np.cumsum([len(s) for s in strings])]).astype(np.uint64)
    data = np.array([v for s in strings for v in s], dtype=np.uint8)
    for p in params:
        cuts, co = oracle.chunk_batch(data, offs, p)
        for f, s in enumerate(strings):
            got = cuts[co[f]:co[f + 1]].tolist()
            assert got == declarative.chunk(s, p), (s, p)


def test_random_inputs_up_to_64_bytes():
    rng = random.Random(2024)
    for _ in range(20000):
        n = rng.randint(0, 64)
        b = [rng.randrange(rng.choice([2, 3, 5, 256])) for _ in range(n)]
        R = rng.randint(2, 6)
        mn = rng.randint(1, 12)
        p = Params(rng.randint(0, 1), R, rng.randint(0, 6), rng.randint(0, 9),
                   mn, rng.randint(mn, 40))
        assert oracle.chunk(_u8(b), p).tolist() == declarative.chunk(b, p)


# ---------------------------------------------------------------------------
# Mutation checks: plausible mistakes planted in a copy of the oracle must be
# caught by the pins above.
# ---------------------------------------------------------------------------
MUTANTS = {
    "trigger_exceeds": ("opp == p->skip_trigger", "opp == p->skip_trigger + 1"),
    "resume_at_j_plus_S": ("i = j + 1 + p->skip_size;", "i = j + p->skip_size;"),
    "no_opp_reset": ("                    opp = 0;\n", ""),
    "scan_from_min": ("p->min_size - R : 0", "p->min_size : 0"),
    "run_counts_pairs": ("if (run == R) return j + 1;", "if (run == R + 1) return j + 1;"),
    "non_strict_target": ("(cur > prev) : (cur < prev)", "(cur >= prev) : (cur <= prev)"),
    "swapped_operands": ("return mode == 0 ? (cur > prev) : (cur < prev);",
                         "return mode == 0 ? (prev > cur) : (prev < cur);"),
    "signed_bytes": ("is_target(p->mode, b[j - 1], b[j])",
                     "is_target(p->mode, (uint8_t)(b[j - 1] ^ 0x80), (uint8_t)(b[j] ^ 0x80))"),
    "cut_before_run_end": ("if (run == R) return j + 1;", "if (run == R) return j;"),
    "no_max_cap": ("(n - c > p->max_size) ? c + p->max_size : n", "n"),
    "run_not_reset": ("            run = 1;\n            if (is_opposing", "            if (is_opposing"),
}


def _pin_suite(chunk):
    """Run the pins against `chunk(bytes, params) -> list`; True if all hold."""
    for name in ("hand_example.json", "trigger_example.json", "vector_example.json"):
        p, b, cuts = _golden(name)
        if chunk(b, p) != cuts:
            return False
    p = oracle.presets(8)
    n = 3 * p.max_size + 5
    if chunk(np.full(n, 9, np.uint8), p) != list(range(p.max_size, n, p.max_size)) + [n]:
        return False
    rng = np.random.default_rng(1)
    b = rng.integers(0, 256, 30000).astype(np.uint8)
    q = Params(0, 4, 0, 0, 40, 400)
    if chunk(b, q) != _no_skip_closed_form(b, q):
        return False
    r = random.Random(3)
    for _ in range(300):
        n = r.randint(0, 40)
        s = [r.randrange(256 if r.random() < 0.5 else 4) for _ in range(n)]
        mn = r.randint(1, 8)
        q = Params(r.randint(0, 1), r.randint(2, 4), r.randint(0, 4), r.randint(0, 5),
                   mn, r.randint(mn, 30))
        if chunk(_u8(s), q) != declarative.chunk(s, q):
            return False
    return True


def _compile_mutant(src_text, tmpdir, name):
    c = os.path.join(tmpdir, name + ".c")
    so = os.path.join(tmpdir, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", "-o", so, c], check=True)
    lib = ctypes.CDLL(so)
    lib.oracle_chunk.restype = ctypes.c_int64
    lib.oracle_chunk.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                 ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]

    def chunk(b, p):
        b = np.ascontiguousarray(b, dtype=np.uint8)
        cap = b.size + 1
        out = np.empty(cap, np.uint64)
        cp = oracle._cparams(p)
        k = lib.oracle_chunk(ctypes.addressof(cp), b.ctypes.data, b.size,
                             out.ctypes.data, cap, None)
        return out[:k].tolist() if k >= 0 else None
    return chunk


def test_pins_hold_for_the_oracle():
    assert _pin_suite(lambda b, p: oracle.chunk(b, p).tolist())


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_mutant(mutant):
    with open(oracle._SRC) as f:
        src = f.read()
    old, new = MUTANTS[mutant]
    assert old in src, "mutation site not found: %s" % mutant
    with tempfile.TemporaryDirectory() as d:
        chunk = _compile_mutant(src.replace(old, new, 1), d, mutant)
        assert not _pin_suite(chunk), "pins did not catch mutant %s" % mutant
