/*
 * seqcdc.h -- C ABI of the GB300 (sm_103a) SeqCDC chunker.
 *
 * SeqCDC (Udayashankar & Al-Kiswany, "Vectorized Sequence-Based Chunking for
 * Data Deduplication") is a content-defined chunking method.  A chunk boundary
 * is placed right after a run of SeqLength strictly increasing (or strictly
 * decreasing) bytes, Sec. III.A.  The first min_size - SeqLength bytes of
 * every chunk are not scanned, Sec. III.B.  Once SkipTrigger byte pairs in the
 * opposite order have been seen, the next SkipSize bytes are skipped,
 * Sec. III.C.  A chunk is cut at max_size when no run completes first,
 * Sec. IV and Sec. VI.  This library computes exactly the boundary list a
 * sequential scan produces, with CUDA kernels over bytes in device memory
 * (or in pinned host memory, read in place over the host link).
 * It has two paths with the same output (see seqcdc_tuning_t.algorithm):
 * a segment map that classifies every byte and resolves the chunk chain
 * across segments, and a chain walk that follows the chain one chunk after
 * the other, many chains at once, reading only the scan windows (the bytes
 * Sec. III.B and III.C leave unread are never loaded).
 *
 * Conventions for every entry point:
 *   - "d_" pointers are CUDA device pointers (or managed memory) that the
 *     caller allocated and owns; the chunking calls also take mapped pinned
 *     host memory for their input and outputs (seqcdc_chunk).  The library never allocates, never frees
 *     and never synchronises the stream, except seqcdc_status() (which
 *     synchronises on purpose).  All work is enqueued on `stream` (a
 *     cudaStream_t passed as void*; NULL = the legacy default stream).
 *   - Input bytes are read-only.  `d_in` / `d_data` must be 16-byte aligned.
 *   - Output cut lists hold chunk END offsets: exclusive, strictly
 *     increasing, the last one equal to the input length.  There is no
 *     leading 0.  Empty input gives an empty list.
 *   - Return values are seqcdc status codes (SEQCDC_OK == 0).  Argument
 *     errors are detected on the host before anything is enqueued.  Errors
 *     that only the device can see (a bounded wait that expired) are
 *     recorded in a status word inside the workspace; read it with
 *     seqcdc_status().
 */
#ifndef SEQCDC_H
#define SEQCDC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SEQCDC_OK         0
#define SEQCDC_EINVAL     1  /* bad parameter set, NULL or misaligned pointer */
#define SEQCDC_ECAPACITY  2  /* output capacity or workspace too small         */
#define SEQCDC_ECUDA      3  /* a CUDA runtime call failed                     */
#define SEQCDC_ETIMEOUT   4  /* a bounded device-side wait expired             */
#define SEQCDC_ERANGE     5  /* input larger than the library supports         */

#define SEQCDC_MODE_INCREASING 0u
#define SEQCDC_MODE_DECREASING 1u

/*
 * Parameter set of Sec. III (modes, SeqLength, SkipTrigger, SkipSize) and the
 * minimum / maximum chunk sizes of Sec. VI.
 *   mode          SEQCDC_MODE_INCREASING or SEQCDC_MODE_DECREASING (Sec. III.A:
 *                 the two modes are exclusive).
 *   seq_length    run length in BYTES (SeqLength); 2..16.  A run of
 *                 seq_length bytes has seq_length-1 strictly ordered pairs.
 *   skip_trigger  number of opposing-order pairs that fires a skip
 *                 (Sec. III.C); 0 disables skipping (the "BASE" variant of
 *                 Sec. VI.D).
 *   skip_size     bytes ignored after a skip fires (Sec. III.C).
 *   min_size      minimum chunk size, >= 1 (Sec. III.B).
 *   max_size      maximum chunk size, >= min_size and <= 131072 (128 KiB:
 *                 one block keeps the bitmaps of its segment plus max_size
 *                 bytes of look-ahead in shared memory).
 */
typedef struct {
    uint32_t mode;
    uint32_t seq_length;
    uint32_t skip_trigger;
    uint32_t skip_size;
    uint64_t min_size;
    uint64_t max_size;
} seqcdc_params_t;

/*
 * Launch tuning (all fields 0 = library default).
 *   segment_bytes  segment map: bytes of input one thread block owns
 *                  (rounded up to a multiple of 1024; at least 4096 and at
 *                  least max_size; lowered if the block's shared memory would
 *                  not fit).  Larger segments mean fewer junctions but more
 *                  shared memory per block.
 *   block_threads  segment map: threads per block of the segment kernel
 *                  (128, 256, 512; any other value means the default).
 *   algorithm      SEQCDC_ALGO_AUTO (0), SEQCDC_ALGO_MAP or SEQCDC_ALGO_WALK.
 *                  AUTO takes the chain walk for batches of at least
 *                  SEQCDC_WALK_MIN_FILES files and for any call of at least
 *                  SEQCDC_WALK_MIN_PIECES full pieces (total_bytes /
 *                  piece_bytes), and the segment map otherwise, except that
 *                  a call whose workspace is too small for the segment map
 *                  but large enough for the chain walk takes the chain walk
 *                  (so a workspace sized for a larger call serves every
 *                  smaller one).  The chain walk needs many chains (pieces)
 *                  at once to be fast; the segment map does not.
 *   piece_bytes    chain walk: bytes of a piece, the unit one warp walks
 *                  (rounded up to a multiple of 64 KiB; at least
 *                  4 x max_size, at most 64 MiB; default 768 KiB, or
 *                  384 x min_size when min_size exceeds 4 KiB, and twice
 *                  that for input read in place from host memory of at
 *                  least 4,096 such doubled pieces).
 */
#define SEQCDC_ALGO_AUTO 0u
#define SEQCDC_ALGO_MAP  1u
#define SEQCDC_ALGO_WALK 2u
#define SEQCDC_WALK_MIN_FILES 256u
#define SEQCDC_WALK_MIN_PIECES 1024u
typedef struct {
    uint32_t segment_bytes;
    uint32_t block_threads;
    uint32_t algorithm;
    uint32_t piece_bytes;
} seqcdc_tuning_t;

/*
 * Fill *out with the segment size, block size and piece size that a chunking
 * call with these parameters and this tuning (NULL or zero fields: library
 * defaults) runs with; out->algorithm is copied from the tuning (AUTO is
 * decided per call, from the number of files).  The defaults are 256 threads,
 * 64 KiB segments (max_size if larger) and 768 KiB pieces (384 x min_size
 * above a 4 KiB min_size).  Returns
 * SEQCDC_EINVAL for an invalid parameter set or a NULL out.
 */
int seqcdc_resolve_tuning(const seqcdc_params_t *p, const seqcdc_tuning_t *tuning,
                          seqcdc_tuning_t *out);

/*
 * Fill *out with the paper's parameters for an expected average chunk size
 * of 4, 8 or 16 KB (Table I for SeqLength / SkipTrigger / SkipSize; Sec. VI
 * for min = 1/2x and max = 2x the expected size, except a 1 KB minimum for
 * 4 KB).  KB = 1024 bytes.  Returns SEQCDC_EINVAL for any other size, a mode
 * other than the two defined ones, or a NULL out.
 */
int seqcdc_params(uint32_t expected_kib, uint32_t mode, seqcdc_params_t *out);

/* SEQCDC_OK if *p is a parameter set this library accepts, else SEQCDC_EINVAL. */
int seqcdc_validate(const seqcdc_params_t *p);

/*
 * Bytes of device workspace seqcdc_chunk_batch() needs for `nfiles` files
 * holding `total_bytes` bytes in all (seqcdc_chunk(): nfiles = 1).  Returns 0
 * for an invalid parameter set.  `tuning` may be NULL.
 */
size_t seqcdc_workspace_size(const seqcdc_params_t *p, uint64_t total_bytes,
                             uint64_t nfiles, const seqcdc_tuning_t *tuning);

/*
 * The path (SEQCDC_ALGO_MAP or SEQCDC_ALGO_WALK) that a chunking call with
 * these arguments takes on input in device memory: seqcdc_chunk() for
 * batch == 0 (nfiles = 1), seqcdc_chunk_batch() otherwise, with a workspace
 * of ws_bytes bytes (input read in place from host memory takes the chain
 * walk under AUTO whenever the workspace holds it).  Returns 0 for an invalid
 * parameter set.  Makes no CUDA call.
 */
int seqcdc_algorithm(const seqcdc_params_t *p, uint64_t total_bytes, uint64_t nfiles,
                     int batch, size_t ws_bytes, const seqcdc_tuning_t *tuning);

/*
 * Chunk one byte stream d_in[0..n).
 *   d_in     device memory, or pinned host memory that is mapped into the
 *            device's address space (cudaHostAlloc / cudaHostRegister; on a
 *            GB300 node every pinned allocation is), which the kernels then
 *            read in place over the host link: AUTO takes the chain walk for
 *            such input when the workspace allows it, and the walk loads
 *            a window 128 bytes at a time from its scan region's start, as
 *            far as the scan reaches, so only a fraction of the bytes cross
 *            (Sec. III.B-C skip the rest).
 *            Pageable host memory gives SEQCDC_EINVAL (after the size
 *            checks, before any launch).  16-byte aligned.
 *   d_cuts   out: up to `cap` uint64 chunk end offsets (device memory, or
 *            mapped pinned host memory that the kernels write to directly;
 *            likewise d_count and, for batches, d_cut_offsets).
 *   cap      capacity of d_cuts in entries; must be >= n / min_size + 1
 *            (always sufficient), else SEQCDC_ECAPACITY.
 *   d_count  out: one uint64, the number of cuts written.
 *   d_ws     workspace of >= seqcdc_workspace_size(p, n, 1, tuning) bytes,
 *            256-byte aligned; its contents need no initialisation.  Two
 *            calls in flight at once must use different workspaces.
 * Asynchronous on `stream`.
 */
int seqcdc_chunk(const seqcdc_params_t *p, const uint8_t *d_in, uint64_t n,
                 uint64_t *d_cuts, uint64_t cap, uint64_t *d_count,
                 void *d_ws, size_t ws_bytes, const seqcdc_tuning_t *tuning,
                 void *stream);

/*
 * Chunk a batch of files laid out back to back in d_data[0..total_bytes)
 * (device memory or mapped pinned host memory, read in place, as d_in of
 * seqcdc_chunk).
 *   d_offsets      nfiles+1 uint64 on the device: file f is
 *                  d_data[d_offsets[f] .. d_offsets[f+1]); d_offsets[0] == 0,
 *                  non-decreasing, d_offsets[nfiles] == total_bytes.
 *   d_cuts         out: cut lists of all files, file after file; the cuts of
 *                  a file are relative to the file's start.
 *   cap            capacity of d_cuts; must be >= total_bytes / min_size +
 *                  nfiles (always sufficient), else SEQCDC_ECAPACITY.
 *   d_cut_offsets  out: nfiles+1 uint64, a CSR index: the cuts of file f are
 *                  d_cuts[d_cut_offsets[f] .. d_cut_offsets[f+1]).
 *   d_ws, ws_bytes as for seqcdc_chunk with (total_bytes, nfiles).
 * Each file is chunked independently, as if it were its own stream.
 * Asynchronous on `stream`.
 */
int seqcdc_chunk_batch(const seqcdc_params_t *p, const uint8_t *d_data,
                       uint64_t total_bytes, const uint64_t *d_offsets,
                       uint64_t nfiles, uint64_t *d_cuts, uint64_t cap,
                       uint64_t *d_cut_offsets, void *d_ws, size_t ws_bytes,
                       const seqcdc_tuning_t *tuning, void *stream);

/*
 * Chunking without any device allocation, for callers that must not allocate:
 * code embedded in a host process whose device memory is owned by another
 * allocator or pool (a storage engine, a framework plugin), and latency-bound
 * paths that cannot afford cudaMalloc / cudaFree, which can synchronise the
 * device and take driver-wide locks.  This entry point has no counterpart in
 * the paper; it is seqcdc_chunk() with its workspace taken from a fixed
 * device array inside this library instead of a caller buffer.
 *
 *   SEQCDC_NOALLOC_SCRATCH_BYTES  size of that array.  It is part of the
 *             library image: every GPU that loads the library holds these
 *             bytes until the process exits.  The input may be at most as
 *             large as fits: the call takes the path whose workspace fits
 *             in it (with AUTO, the chain walk where the segment map's would
 *             not), and that workspace must not exceed it, else
 *             SEQCDC_ERANGE is returned before anything runs.  With the
 *             paper's parameter sets that is up to about 1 GiB of input at
 *             the 4 KB setting, 4 GiB at 8 KB and 8 GiB at 16 KB.
 *   d_in, n, d_cuts, cap, d_count, tuning, stream  as for seqcdc_chunk().
 *   d_status  optional (may be NULL): one uint32 on the device that receives
 *             the call's device-side status (SEQCDC_OK, SEQCDC_ETIMEOUT or
 *             SEQCDC_ECAPACITY), written on `stream` after the chunking.
 * It calls no cudaMalloc, cudaFree or other allocating routine.  The first
 * call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.
 * A cudaDeviceReset() unloads the library's device image and invalidates
 * that address: do not use this entry point after one in the same process.
 * All calls share the one array and it keeps the last call's contents (the
 * kernels reset what they need): calls that overlap on the GPU -- from two
 * streams or two host threads without ordering -- race and give wrong results.
 */
#define SEQCDC_NOALLOC_SCRATCH_BYTES (16u << 20)
int seqcdc_chunk_noalloc(const seqcdc_params_t *p, const uint8_t *d_in,
                         uint64_t n, uint64_t *d_cuts, uint64_t cap,
                         uint64_t *d_count, uint32_t *d_status,
                         const seqcdc_tuning_t *tuning, void *stream);

/*
 * Synchronise `stream`, then return the device-side status recorded in d_ws by
 * the last call that used it: SEQCDC_OK, SEQCDC_ETIMEOUT when a bounded
 * wait inside a kernel expired, or SEQCDC_ECAPACITY when the device found more
 * cuts than `cap` (both mean the outputs are not valid).  Returns
 * SEQCDC_ECUDA if the synchronisation itself fails.
 */
int seqcdc_status(const void *d_ws, void *stream);

/*
 * Copy n byte ranges, in order, each as one cudaMemcpyAsync on `stream`:
 * dst[dst_off[i] .. dst_off[i] + len[i]) = src[src_off[i] .. + len[i]).
 * dst and src are device memory or pinned host memory (any direction);
 * dst_off, src_off and len are host arrays of n entries; ranges of length 0
 * are skipped.  A batch of many requests is gathered into one buffer this
 * way (the serving loop) without a runtime call per request from the
 * caller's language.  Returns SEQCDC_EINVAL for n > 0 with a NULL pointer
 * or array, SEQCDC_ECUDA if a copy cannot be enqueued (the copies before it
 * stay enqueued).
 */
int seqcdc_copy_ranges(void *dst, const void *src, const uint64_t *dst_off,
                       const uint64_t *src_off, const uint64_t *len, uint64_t n,
                       void *stream);

/*
 * Synchronise `stream` and copy up to `n` (<= 8) path counters of the last
 * call that used d_ws into out[].  Segment map: [0] segments processed,
 * [1] segments whose natural entries could not all be walked, [2] segments
 * with more distinct exits than the library publishes, [3] look-backs that
 * had to wait for a predecessor's true exit, [4] segments found inconsistent
 * by the verify pass, [5] segments re-chunked by the repair passes,
 * [6] segments the resolve pass emitted from a guessed entry (or could not
 * emit) because their true entry was unknown or not one of their natural
 * cuts, [7] total look-back depth.  Chain walk: [0] pieces walked, [1] chunks
 * found by the piece walks, [2] junction walks, [3] chunks the junction walks
 * took before meeting their piece's walk, [4] junction walks that left their
 * piece without meeting it, [5] pieces found inconsistent, [6] junction walks
 * redone by the repair pass, [7] 1 KiB windows the piece walks loaded (32-byte
 * sectors for input read in place from host memory).  The
 * counters describe which code paths ran; the output is exact either way.
 */
int seqcdc_stats(const void *d_ws, void *stream, uint32_t *out, uint32_t n);

/*
 * Bound, in nanoseconds, on every device-side wait of the chunking calls made
 * later from this host thread; returns the previous bound.  The default is
 * SEQCDC_DEFAULT_WAIT_NS (2 s).  Only the segment map waits: its resolve pass
 * finds each segment's true entry by decoupled look-back, which waits for a
 * preceding segment to publish its exit (the chain of Sec. III is sequential,
 * so a segment's first chunk depends on where the previous segment's last
 * chunk ends).  A wait that outlasts the bound gives up: the kernel records
 * SEQCDC_ETIMEOUT in the workspace status (read it with seqcdc_status) and
 * finishes without that value, so the call ends and the CUDA context stays
 * usable, but the outputs of that call are not valid.  A bound of 0 gives up
 * at the first check that finds the value missing.  Calls on other host
 * threads are not affected.  Allocates nothing; makes no CUDA call.
 */
#define SEQCDC_DEFAULT_WAIT_NS 2000000000ull
uint64_t seqcdc_set_wait_limit_ns(uint64_t ns);

/*
 * Measurement hook: record the CUDA events `ev_begin` / `ev_end` (cudaEvent_t
 * passed as void*) on the call's stream immediately before and after the
 * dominant kernel (the segment kernel of the segment map, the piece-walk
 * kernel of the chain walk) of every later seqcdc_chunk / seqcdc_chunk_batch
 * call made from this host thread, so that its device time can be read with
 * cudaEventElapsedTime.  A call made while its stream is being captured into
 * a CUDA graph records them as external event nodes, which fire on every
 * launch of the graph.  Pass NULL, NULL to stop.  The events are owned by the
 * caller.  Always returns SEQCDC_OK.
 */
int seqcdc_profile_events(void *ev_begin, void *ev_end);

/*
 * Fingerprinting and deduplication: the step after chunking (Sec. II).  These
 * entry points take the output of seqcdc_chunk_batch() (for one stream: one
 * file, d_offsets = {0, n}, d_cut_offsets = {0, count}).
 *
 * seqcdc_fingerprint_batch: SHA-256 (FIPS 180-4) of every chunk.
 *   d_data, total_bytes, d_offsets, nfiles  as for seqcdc_chunk_batch()
 *             (d_data 16-byte aligned, nfiles >= 1).
 *   d_cuts, d_cut_offsets, ncuts  the chunking output; ncuts = the number of
 *             cuts (d_cut_offsets[nfiles]); chunk i of file f is
 *             [d_offsets[f] + previous cut of f (or 0), d_offsets[f] + d_cuts[i]).
 *   d_digests out: 32 bytes per chunk, the digest in its standard byte order
 *             (4-byte aligned).
 *   d_sizes   out, optional (NULL): chunk sizes in bytes, one uint32 each.
 * Asynchronous on `stream`.  SEQCDC_EINVAL for NULL or misaligned pointers,
 * SEQCDC_ERANGE for 2^32 or more chunks.
 */
int seqcdc_fingerprint_batch(const uint8_t *d_data, uint64_t total_bytes,
                             const uint64_t *d_offsets, uint64_t nfiles,
                             const uint64_t *d_cuts, const uint64_t *d_cut_offsets,
                             uint64_t ncuts, uint8_t *d_digests, uint32_t *d_sizes,
                             void *stream);

/* Bytes of the hash table seqcdc_dedup() needs for `nchunks` chunks. */
size_t seqcdc_dedup_table_bytes(uint64_t nchunks);

/*
 * Count the distinct chunks among `nchunks` fingerprints (32-byte digests from
 * seqcdc_fingerprint_batch, with their sizes): d_out[0] = distinct chunks,
 * d_out[1] = their bytes (so the savings of Eq. 1 are 1 - d_out[1] / all
 * bytes).  Chunks with equal digests are the same chunk.  d_table: caller
 * workspace of >= seqcdc_dedup_table_bytes(nchunks) bytes (4-byte aligned),
 * no initialisation needed.  Asynchronous on `stream`.
 */
int seqcdc_dedup(const uint8_t *d_digests, const uint32_t *d_sizes, uint64_t nchunks,
                 void *d_table, size_t table_bytes, uint64_t *d_out, void *stream);

/* Static, human-readable text for a status code. */
const char *seqcdc_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* SEQCDC_H */
