/*
 * Plain, single-threaded CPU SeqCDC -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the oracle the GPU path is checked against.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it; the library's product path never does.  It shares no code, header or
 * constant with the CUDA implementation.
 *
 * What it computes (Udayashankar & Al-Kiswany, "Vectorized Sequence-Based
 * Chunking for Data Deduplication", Sec. III):
 *   - Sec. III.A: a boundary is placed right after a run of SeqLength bytes
 *     that is strictly increasing (Increasing mode) or strictly decreasing
 *     (Decreasing mode); bytes are unsigned values 0..255.
 *   - Sec. III.B: the first (min_size - SeqLength) bytes of every chunk are
 *     not scanned, so no chunk ends before min_size.
 *   - Sec. III.C: byte pairs in the order opposite to the target are counted;
 *     when the count reaches SkipTrigger the next SkipSize bytes are ignored
 *     and both counters restart.
 *   - Sec. IV ("Maximum chunk size") / Sec. VI: a chunk is cut at max_size
 *     when no run completes first; the last chunk ends at the input end.
 *
 * The scan is a byte-at-a-time loop over the pair (b[j-1], b[j]), written in
 * the order the paper describes the steps.  Readings of points the paper
 * leaves open are fixed as follows (each one is a plain choice, listed again
 * in the design notes):
 *   - run length counts BYTES: SeqLength bytes = SeqLength-1 strict pairs
 *     (the vector description of Sec. III.D declares the boundary SeqLength
 *     bytes after the first byte of the run);
 *   - comparisons are strict and unsigned; an equal pair is neither a target
 *     nor an opposing pair and breaks the run;
 *   - the skip fires when the opposing count REACHES SkipTrigger
 *     (Sec. III.C "When SkipTrigger pairs ... are detected");
 *     SkipTrigger == 0 disables skipping (the BASE variant of Sec. VI.D);
 *   - after the pair (j-1, j) fires the skip, bytes j+1 .. j+SkipSize are
 *     ignored and the next run starts at byte j+1+SkipSize;
 *   - the pair straddling the sub-minimum region, the pair straddling a
 *     skipped region and the pair straddling a cut are never examined;
 *   - a forced cut at chunk_start + max_size happens whenever no run
 *     completes before it, even when a skip jumped past it.
 *
 * Every function here is parity-pinned by the CPU tests: a hand-worked
 * example, the vector example of Sec. III.D, closed forms, invariants and a
 * second, independently written prefix-count formulation.
 */
#include <stddef.h>
#include <stdint.h>

/* Parameter set of Sec. III / Table I, laid out field by field. */
typedef struct {
    uint32_t mode;          /* 0 = Increasing, 1 = Decreasing            */
    uint32_t seq_length;    /* SeqLength, in bytes                        */
    uint32_t skip_trigger;  /* SkipTrigger; 0 = never skip                */
    uint32_t skip_size;     /* SkipSize, bytes ignored after a trigger    */
    uint64_t min_size;      /* minimum chunk size                         */
    uint64_t max_size;      /* maximum chunk size                         */
} oracle_params_t;

enum { ORACLE_OK = 0, ORACLE_EINVAL = -1, ORACLE_ECAPACITY = -2 };

static int oracle_params_valid(const oracle_params_t *p)
{
    if (!p) return 0;
    if (p->mode > 1) return 0;
    if (p->seq_length < 2 || p->seq_length > 16) return 0;
    if (p->min_size < 1 || p->max_size < p->min_size) return 0;
    return 1;
}

/* Target order of Sec. III.A: the later byte is strictly above (Increasing)
 * or strictly below (Decreasing) the earlier one. */
static int is_target(uint32_t mode, uint8_t prev, uint8_t cur)
{
    return mode == 0 ? (cur > prev) : (cur < prev);
}

/* Opposing order of Sec. III.C: the strict reverse of the target order. */
static int is_opposing(uint32_t mode, uint8_t prev, uint8_t cur)
{
    return mode == 0 ? (cur < prev) : (cur > prev);
}

/*
 * One chunk: scan from chunk start c and return its end offset (exclusive).
 * `examined` (may be NULL) accumulates the number of byte pairs looked at.
 */
static uint64_t oracle_one_chunk(const oracle_params_t *p, const uint8_t *b,
                                 uint64_t n, uint64_t c, uint64_t *examined)
{
    const uint64_t R = p->seq_length;
    uint64_t limit = (n - c > p->max_size) ? c + p->max_size : n;
    /* Sec. III.B: the first (min - SeqLength) bytes are not scanned. */
    uint64_t i = c + ((p->min_size > R) ? p->min_size - R : 0);
    uint64_t run = 1;  /* bytes in the current target-order run, from i  */
    uint64_t opp = 0;  /* opposing pairs since the last (re)start        */
    uint64_t j = i + 1;
    while (j < limit) {
        if (examined) (*examined)++;
        if (is_target(p->mode, b[j - 1], b[j])) {
            run++;
            if (run == R) return j + 1;    /* boundary right after the run */
        } else {
            run = 1;
            if (is_opposing(p->mode, b[j - 1], b[j])) {
                opp++;
                if (p->skip_trigger != 0 && opp == p->skip_trigger) {
                    /* Sec. III.C: ignore the next SkipSize bytes, reset. */
                    i = j + 1 + p->skip_size;
                    run = 1;
                    opp = 0;
                    j = i + 1;
                    continue;
                }
            }
        }
        j++;
    }
    return limit;  /* forced cut at c + max_size, or the input end */
}

/*
 * Chunk b[0..n) and write the chunk END offsets (strictly increasing, the last
 * one equal to n; none for n == 0) into cuts[0..cap).  Returns the number of
 * cuts, ORACLE_EINVAL for a bad parameter set, ORACLE_ECAPACITY when cap is
 * too small.  `examined` (may be NULL) receives the number of byte pairs the
 * scan compared.
 */
int64_t oracle_chunk(const oracle_params_t *p, const uint8_t *b, uint64_t n,
                     uint64_t *cuts, uint64_t cap, uint64_t *examined)
{
    if (!oracle_params_valid(p)) return ORACLE_EINVAL;
    if (examined) *examined = 0;
    uint64_t count = 0;
    uint64_t c = 0;
    while (c < n) {
        uint64_t e = oracle_one_chunk(p, b, n, c, examined);
        if (count >= cap) return ORACLE_ECAPACITY;
        cuts[count++] = e;
        c = e;
    }
    return (int64_t)count;
}

/*
 * Files laid out back to back: file f is b[offsets[f] .. offsets[f+1]).
 * Each file is chunked on its own; its cuts (relative to the file start) go to
 * cuts[cut_offsets[f] .. cut_offsets[f+1]).  cut_offsets has nfiles+1 entries.
 * Returns the total number of cuts or a negative status.
 */
int64_t oracle_chunk_batch(const oracle_params_t *p, const uint8_t *b,
                           const uint64_t *offsets, uint64_t nfiles,
                           uint64_t *cuts, uint64_t cap, uint64_t *cut_offsets)
{
    if (!oracle_params_valid(p)) return ORACLE_EINVAL;
    uint64_t total = 0;
    for (uint64_t f = 0; f < nfiles; f++) {
        cut_offsets[f] = total;
        if (offsets[f + 1] < offsets[f]) return ORACLE_EINVAL;
        int64_t k = oracle_chunk(p, b + offsets[f], offsets[f + 1] - offsets[f],
                                 cuts + total, cap - total, NULL);
        if (k < 0) return k;
        total += (uint64_t)k;
    }
    cut_offsets[nfiles] = total;
    return (int64_t)total;
}
