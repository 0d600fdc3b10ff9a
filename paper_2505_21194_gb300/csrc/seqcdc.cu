// seqcdc.cu -- SeqCDC chunking on GB300 (sm_103a): kernels and the C ABI.
//
// What is computed (Udayashankar & Al-Kiswany, "Vectorized Sequence-Based
// Chunking for Data Deduplication"):
//   Sec. III.A  a chunk ends right after SeqLength bytes in strictly increasing
//               (Increasing mode) or strictly decreasing (Decreasing mode)
//               order; bytes are unsigned.
//   Sec. III.B  the first min_size - SeqLength bytes of a chunk are not scanned.
//   Sec. III.C  opposing-order pairs are counted from the start of a scan
//               region; when the count reaches SkipTrigger the next SkipSize
//               bytes are ignored and both counters restart.
//   Sec. IV/VI  a chunk is cut at max_size if no run completes first.
// The scan of Sec. III.D is evaluated on bitmaps: T[j] marks a target-order
// pair (b[j-1], b[j]), O[j] an opposing pair, and
// E[j] = T[j] & T[j-1] & ... & T[j-SeqLength+2] marks the last byte of a
// boundary run (the AND of SeqLength-1 shifted comparison masks of
// Sec. III.D).  A scan region starting at byte i ends at the first E bit at or
// after i + SeqLength - 1 (cut right after it) or at the SkipTrigger-th O bit
// after i (skip), whichever comes first -- the first-set-bit and n-th-set-bit
// queries of Sec. III.D.
//
// Parallel structure (the paper scans one stream sequentially):
//   plan     split every file into segments ("items") of L bytes.
//   segment  one thread block per item.  The block builds the E and O bitmaps
//            of its L bytes plus max_size bytes of look-ahead in shared memory
//            (SWAR byte compares, 16 bytes per thread step) with per-256-byte
//            summaries, then walks the chunk chain from EVERY natural cut
//            (E bit + 1) in the item's first max_size bytes, merging chains
//            that meet at a common cut.  Each entry thus maps to an exit (the
//            first cut at or after the item end).  The block publishes the set
//            of distinct exits ("image", <= 32 values), then the map from its
//            predecessor's image to its own exits (a <= 32-entry function),
//            and finds its true entry by decoupled look-back: composing
//            predecessors' maps until one that has published its true exit.
//            It then emits its cuts from shared memory.
//   verify   check entry[s] == exit[s-1] along every file (by induction from
//            the file start the output is then exact); a repair pass
//            re-chunks from the first inconsistent item (needed only when a
//            forced cut at max_size entered an item away from its natural
//            entries, e.g. inside long runs of equal bytes).
//   compact  exclusive scan of per-item cut counts and copy into the
//            caller's CSR output.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "seqcdc.h"
#include "common.cuh"
#include "walk.h"

namespace {

// ---------------------------------------------------------------------------
// Limits and layout constants.
// ---------------------------------------------------------------------------
constexpr uint32_t kCandPerLane = 3;  // chunk-step candidates per lane (map kernel)
constexpr int kImgHash = 128;      // distinct-exit hash slots (power of two)
constexpr int kMaxImage = 32;      // distinct exits published per item (one per lane)
constexpr int kFileTile = 1024;    // files per plan block
constexpr int kItemTile = 256;     // items per compaction tile
constexpr int kEmitSplit = 8;      // emit blocks per compaction tile
constexpr uint32_t kMaxSeqLength = 16;
constexpr uint64_t kMaxMaxSize = 131072;
constexpr uint64_t kWaitNs = SEQCDC_DEFAULT_WAIT_NS;  // default bound on a device wait

// Item state bits (set once, in this order of availability).
constexpr uint32_t F_IMG = 1u;     // image (distinct exits) published
constexpr uint32_t F_NOIMG = 2u;   // no image (more than kMaxImage exits)
constexpr uint32_t F_AGG = 4u;     // map predecessor image -> exits published
constexpr uint32_t F_NOAGG = 8u;   // no such map (predecessor had no image)
constexpr uint32_t F_INCL = 16u;   // true exit, entry and cuts published
constexpr uint32_t F_RUN = 32u;    // first item of a run of inconsistent items
// Rounds of verify + parallel run repair before the sequential fallback.
constexpr uint32_t kRepairRounds = 2;

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kTerminal = 0x80000000u;  // candidate next: first cut >= item end
constexpr uint32_t kEscape = 0xFFFFFFFFu;    // candidate next: forced cut inside item
constexpr uint32_t kAbnormal = 0xFFFFFFFFu;  // cand_n: too many natural cuts
constexpr uint64_t kBad = ~0ull;             // unknown exit / entry

// Workspace header (first 256 bytes of the workspace).
struct WsHeader {
  uint32_t status;
  uint32_t ticket;
  uint32_t nitems;
  uint32_t stats[8];  // see seqcdc_stats()
  uint32_t nruns[kRepairRounds];  // runs of inconsistent items found by each verify round
  uint32_t runq[kRepairRounds];   // run queue head of each parallel repair round
  uint32_t pad[53 - 2 * kRepairRounds];
};

enum : uint32_t {
  ST_ITEMS = 0,         // items resolved
  ST_ABNORMAL = 1,      // items with more natural cuts than tabulated
  ST_NOIMG = 2,         // items without a published exit set
  ST_LB_WAITS = 3,      // look-backs that had to wait for a true exit
  ST_INCONSISTENT = 4,  // items whose entry disagreed with the predecessor
  ST_RECOMPUTED = 5,    // items re-chunked by the repair pass
  ST_REPLAYED = 6,      // items the resolve kernel emitted from a guessed entry (or could not emit)
  ST_LB_STEPS = 7,      // total look-back depth
};

struct Layout {
  size_t hdr, seg_base, ftile, state, incl, entry, first_bad, count, img_n,
      img, agg, cand_n, ent_n, cand_pos, cand_nxt, ent_term, slot, itile, runs, item_file,
      total;
  uint64_t imax;     // upper bound on items
  uint64_t nftiles;  // plan tiles
  uint64_t nitiles;  // compaction tiles
  uint32_t L;        // segment bytes
  uint32_t slot_cap; // cuts per item slot
};

struct Geom {
  const uint8_t *data;
  uint64_t total;
  const uint64_t *offsets;  // nullptr: single stream of `total` bytes
  uint64_t nfiles;
  uint32_t L;
  uint32_t cap;             // natural cuts tabulated per item (L / 64)
  uint64_t wait_ns;         // bound on each device-side wait (ns)
  uint32_t host;            // data is pinned host memory (no bulk L2 prefetch of it)
};

// Natural cuts tabulated per item: one per 96 bytes.  Uniform random input
// has one per ~125 bytes at SeqLength 5 (526 +- 26 per 64 KiB; the
// benchmark's 10,000 files reach at most 630 per 64 KiB item); an item with
// more goes to the repair pass.
__host__ __device__ inline uint32_t cand_cap(uint32_t L) { return L / 96 < 256 ? 256 : L / 96; }

__host__ __device__ inline uint64_t file_start(const Geom &g, uint64_t f) {
  return g.offsets ? g.offsets[f] : 0;
}
__host__ __device__ inline uint64_t file_size(const Geom &g, uint64_t f) {
  return g.offsets ? g.offsets[f + 1] - g.offsets[f] : g.total;
}

struct WsPtrs {
  WsHeader *hdr;
  uint32_t *seg_base;   // nfiles + 1: first item of each file
  uint32_t *ftile;      // per plan tile
  uint32_t *state;      // per item
  uint64_t *incl;       // per item: exit from `entry` (file-relative)
  uint64_t *entry;      // per item: entry the item's cuts were computed from
  uint32_t *first_bad;  // per file: first inconsistent item (verify pass)
  uint32_t *count;      // per item: cuts emitted
  uint32_t *img_n;      // per item: image size
  uint64_t *img;        // per item x kMaxImage: distinct exits (file-relative)
  uint64_t *agg;        // per item x kMaxImage: exit for each predecessor image value
  uint32_t *cand_n;     // per item: natural cuts tabulated (kAbnormal: too many)
  uint32_t *ent_n;      // per item: how many of them are entries (< p_s + max)
  uint32_t *cand_pos;   // per item x kMaxCand: positions (relative to the item start)
  uint32_t *cand_nxt;   // per item x kMaxCand: next candidate / terminal / escape
  uint32_t *ent_term;   // per item x kMaxCand: exit of each entry (relative) or escape
  uint64_t *slot;       // per item x slot_cap (file-relative cuts)
  uint32_t *itile;      // per compaction tile
  uint32_t *runs;       // per item: first items of runs to repair (verify rounds)
  uint32_t *item_file;  // per item: its file (written by the map kernel)
  uint32_t slot_cap;
};

// ---------------------------------------------------------------------------
// Small device helpers.
// ---------------------------------------------------------------------------

// Wait until (*flag & mask) != 0, at most limit_ns.  Returns the flag value,
// or 0 after recording SEQCDC_ETIMEOUT in the workspace status.
__device__ uint32_t wait_any(const uint32_t *flag, uint32_t mask, WsHeader *hdr,
                             uint64_t limit_ns) {
  uint32_t v = ld_acquire(flag);
  if (v & mask) return v;
  const uint64_t t0 = global_ns();
  uint32_t backoff = 32;
  for (uint64_t it = 0; it < (1ull << 32); ++it) {
    __nanosleep(backoff);
    if (backoff < 512) backoff <<= 1;
    v = ld_acquire(flag);
    if (v & mask) return v;
    if (global_ns() - t0 > limit_ns) break;
  }
  atomicExch(&hdr->status, (uint32_t)SEQCDC_ETIMEOUT);
  return 0;
}

// ---------------------------------------------------------------------------
// Bitmaps of one item in shared memory.  Positions are relative to the window
// base B (file-relative): rel = pos - B; word w covers rel 32w .. 32w+31.
//   E, O   run-end and opposing-pair bits
//   nz     bit w of the mask: E[w] != 0
//   sbE, sbO  E and O bits in the words before each step of 64 words
//   locO   O bits in the words of w's step before w
// A scan-region query (Sec. III.D: first set bit of the combined run mask;
// position of the SkipTrigger-th opposing pair) is a few lookups: the first
// run end from the nonzero mask, the opposing pairs before it from the O
// counts, and, when there are SkipTrigger of them, their position by a
// binary search over the counts of the words in between.
// ---------------------------------------------------------------------------
struct Bits {
  const uint32_t *E;
  const uint32_t *O;
  const uint32_t *nz;
  const uint32_t *sbO;
  const uint16_t *locO;
  uint32_t W;
};

// O bits in the words before w.
__device__ __forceinline__ uint32_t o_before_word(const Bits &b, uint32_t w) {
  return b.sbO[w >> 6] + b.locO[w];
}

// O bits at rel positions before x (x < 32 W).
__device__ __forceinline__ uint32_t o_before(const Bits &b, uint32_t x) {
  const uint32_t w = x >> 5;
  return o_before_word(b, w) + __popc(b.O[w] & ((1u << (x & 31)) - 1u));
}

// One scan region of the chunker (Sec. III.A-C) from scan position i with
// chunk limit lim: returns the cut (run end + 1 when a run completes before
// the SkipTrigger-th opposing pair; lim when the chunk reaches its maximum
// size or the input end), or kNone after moving i past a content-defined skip.
// Every index is clamped into the window, so lanes without work (lim = 0,
// result lim) run the same instructions.
__device__ __forceinline__ uint32_t region_step(const Bits &b, const DevParams &p,
                                                uint32_t &i, uint32_t lim) {
  const uint32_t Wm1 = b.W - 1;
  const bool open = i + 1 < lim;
  // e: the first E bit at or after i + SeqLength - 1, if below lim.
  uint32_t e = kNone;
  {
    const uint32_t xs = i + p.R - 1;
    uint32_t w = min(xs >> 5, Wm1);
    uint32_t m = b.E[w] & (~0u << (xs & 31));
    if (!m && open) {
      const uint32_t w1 = w + 1;
      if ((w1 << 5) < lim) {
        uint32_t q = w1 >> 5;
        uint32_t z = b.nz[q] & (~0u << (w1 & 31));
        while (!z && ((q + 1) << 10) < lim) z = b.nz[++q];
        if (z) {
          w = (q << 5) + (__ffs(z) - 1);
          m = b.E[w];
        }
      }
    }
    if (m && xs < lim) {
      const uint32_t pos = (w << 5) + (__ffs(m) - 1);
      if (pos < lim) e = pos;
    }
  }
  // No run end before lim: no later region can cut either.
  if (!open || e == kNone) return lim;  // maximum size or end of input (Sec. IV)
  if (p.T == 0) return e + 1;           // skipping disabled
  // Opposing pairs in [i + 1, e): fewer than SkipTrigger means the run ends
  // first.
  const uint32_t x = i + 1;
  const uint32_t rx = o_before(b, x);
  if (o_before(b, e) - rx < p.T) return e + 1;  // boundary run (Sec. III.A)
  // The skip point: O bit number t = rx + SkipTrigger (from 1), in the last
  // word w of [x / 32, e / 32] whose preceding count is below t.
  const uint32_t t = rx + p.T;
  uint32_t lo = x >> 5, hi = e >> 5;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (o_before_word(b, mid) < t) lo = mid; else hi = mid - 1;
  }
  const uint32_t sp = (lo << 5) + nth_set_bit(b.O[lo], t - o_before_word(b, lo));
  i = sp + 1 + p.S;                     // content-defined skip (Sec. III.C)
  return kNone;
}

// One chunk: from chunk start c (rel) return its end (rel).  `end_rel` is the
// rel position of the file end.
__device__ uint32_t chunk_step(const Bits &b, const DevParams &p, uint32_t c,
                               uint32_t end_rel) {
  const uint32_t lim = (end_rel - c > p.mx) ? c + p.mx : end_rel;
  uint32_t i = c + (p.mn > p.R ? p.mn - p.R : 0u);
  while (true) {
    const uint32_t y = region_step(b, p, i, lim);
    if (y != kNone) return y;
  }
}

// ---------------------------------------------------------------------------
// Plan: seg_base[f] = sum of ceil(n_g / L) over g < f; item count.
// ---------------------------------------------------------------------------
__global__ void plan_tiles_kernel(Geom g, WsPtrs ws) {
  __shared__ uint32_t red[32];
  const uint64_t f0 = (uint64_t)blockIdx.x * kFileTile;
  uint32_t sum = 0;
  for (uint64_t f = f0 + threadIdx.x; f < f0 + kFileTile && f < g.nfiles;
       f += blockDim.x) {
    sum += (uint32_t)((file_size(g, f) + g.L - 1) / g.L);
  }
  for (int d = 16; d; d >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    ws.ftile[blockIdx.x] = s;
  }
}

__global__ void plan_scan_kernel(Geom g, WsPtrs ws, uint64_t nftiles,
                                 uint64_t imax) {
  __shared__ uint32_t scratch[32];
  __shared__ uint32_t s_prefix;
  uint32_t part = 0;
  for (uint64_t t = threadIdx.x; t < blockIdx.x; t += blockDim.x) part += ws.ftile[t];
  for (int d = 16; d; d >>= 1) part += __shfl_down_sync(0xffffffffu, part, d);
  if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += scratch[w];
    s_prefix = s;
  }
  __syncthreads();
  uint32_t running = s_prefix;
  const uint64_t f0 = (uint64_t)blockIdx.x * kFileTile;
  for (uint64_t c0 = f0; c0 < f0 + kFileTile; c0 += blockDim.x) {
    const uint64_t f = c0 + threadIdx.x;
    const bool live = f < g.nfiles && f < f0 + kFileTile;
    const uint32_t v = live ? (uint32_t)((file_size(g, f) + g.L - 1) / g.L) : 0u;
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, scratch, &tot);
    if (live) ws.seg_base[f] = running + ex;
    running += tot;
  }
  if (blockIdx.x == nftiles - 1 && threadIdx.x == 0) {
    ws.seg_base[g.nfiles] = running;
    ws.hdr->nitems = running;
    ws.hdr->ticket = 0;
    ws.hdr->status = 0;
    for (int k = 0; k < 8; ++k) ws.hdr->stats[k] = 0;
    for (uint32_t k = 0; k < kRepairRounds; ++k) ws.hdr->nruns[k] = ws.hdr->runq[k] = 0;
  }
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < imax;
       i += (uint64_t)gridDim.x * blockDim.x) {
    ws.state[i] = 0;
  }
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < g.nfiles;
       f += (uint64_t)gridDim.x * blockDim.x) {
    ws.first_bad[f] = 0xffffffffu;
  }
}

// ---------------------------------------------------------------------------
// Per-item machinery.
// ---------------------------------------------------------------------------
// Geometry of one item: segment `seg` of a file.
struct SegGeom {
  int64_t B;          // window base (file-relative); global index of rel 0 is 16-aligned
  uint64_t p_s, q_s;  // the item's bytes [p_s, q_s) (file-relative)
  uint64_t n_f;       // file size
  uint64_t gbase;     // global index of the file's first byte
  uint32_t W;         // bitmap words of the window [B, B + 32 W)
  uint32_t seg;
};

struct SegShared {
  SegGeom gm;
  uint64_t exit;      // repair: exit of the item just re-chunked
  uint32_t flag;      // repair: broadcast from thread 0
  uint32_t nc, nent, ninvalid, nimg, qhead;
  uint32_t scratch[32];
};

// Shared memory of the map kernel (bitmaps, query tables, candidate graph).
struct MapSmem {
  uint32_t *O;       // o_words(W)
  uint32_t *E;       // W + 1
  uint32_t *nz;      // nz_words(W)
  uint32_t *sbE;     // W / 64 + 2
  uint32_t *sbO;     // W / 64 + 2
  uint32_t *cpos;    // cap: candidate positions (rel)
  uint32_t *cnxt;    // cap: next candidate index or terminal code
  uint32_t *ihash;   // kImgHash: distinct exits
  uint32_t *bscratch;  // 64: block helpers
  uint16_t *locO;    // W + 2
  uint16_t *erank_c; // L / 32 + 4: index of each candidate-range word's first candidate
};

// Words of the nonzero-E mask: one bit per bitmap word, whole 64-word steps.
__host__ __device__ inline uint32_t nz_words(uint32_t W) { return ((W + 63) >> 6) * 2 + 2; }
// O words: whole groups of four, plus one spare group.
__host__ __device__ inline uint32_t o_words(uint32_t W) { return ((W + 3) & ~3u) + 4; }

__device__ __forceinline__ MapSmem carve(unsigned char *raw, uint32_t W, uint32_t L) {
  const uint32_t cap = cand_cap(L);
  MapSmem m;
  m.O = reinterpret_cast<uint32_t *>(raw);  // 16-byte aligned
  m.E = m.O + o_words(W);
  m.nz = m.E + W + 1;
  m.sbE = m.nz + nz_words(W);
  m.sbO = m.sbE + (W >> 6) + 2;
  m.cpos = m.sbO + (W >> 6) + 2;
  m.cnxt = m.cpos + cap;
  m.ihash = m.cnxt + cap;
  m.bscratch = m.ihash + kImgHash;
  m.locO = reinterpret_cast<uint16_t *>(m.bscratch + 64);
  m.erank_c = m.locO + W + 2;
  return m;
}

__host__ __device__ inline size_t map_smem_bytes(uint32_t W, uint32_t L) {
  const uint32_t cap = cand_cap(L);
  return (size_t)4 * (o_words(W) + (W + 1) + nz_words(W) + 2 * ((W >> 6) + 2) +
                      2 * (size_t)cap + kImgHash + 64) +
         (size_t)2 * ((W + 2) + (L / 32 + 4)) + 16;
}

// The file of an item (largest f with seg_base[f] <= item), by one warp: a
// 32-ary search (three rounds cover 32768 files).
__device__ uint32_t find_file_warp(const uint32_t *seg_base, uint64_t nfiles,
                                   uint32_t item) {
  const int lane = threadIdx.x & 31;
  uint64_t lo = 0, hi = nfiles;  // answer in [lo, hi); seg_base[lo] <= item
  while (hi - lo > 1) {
    const uint64_t step = (hi - lo + 31) / 32;
    const uint64_t probe = lo + (uint64_t)lane * step;
    const bool ok = probe < hi && seg_base[probe] <= item;
    const uint32_t m = __ballot_sync(0xffffffffu, ok);
    const uint64_t nlo = lo + (uint64_t)(31 - __clz(m)) * step;
    hi = min(nlo + step, hi);
    lo = nlo;
  }
  return (uint32_t)lo;
}

// The file end relative to the window base, for chunk limits.  A file can be
// far longer than 4 GiB; any value past the window (at most L + max_size + 64
// bytes long) gives the same limits, so it is clamped to 32 bits.
__device__ __forceinline__ uint32_t end_rel_of(uint64_t n_f, int64_t B) {
  const int64_t r = (int64_t)n_f - B;
  return r >= (int64_t)0xffffffffLL ? 0xffffffffu : (uint32_t)r;
}

// Ask L2 for the input bytes [lo, hi) (global byte indices, clamped to the
// input and to 16-byte boundaries) with bulk prefetches of up to 64 KiB, one
// per lane of the calling warp: the block's loads that follow then find them
// in L2 instead of each load step waiting for HBM.
__device__ __forceinline__ void prefetch_l2(const uint8_t *base, int64_t lo, int64_t hi,
                                            uint64_t total) {
  if (lo < 0) lo = 0;
  if (hi > (int64_t)total) hi = (int64_t)total;
  lo = (lo + 15) & ~(int64_t)15;
  hi &= ~(int64_t)15;
  const int64_t lane = threadIdx.x & 31;
  for (int64_t a = lo + lane * 65536; a < hi; a += 32 * 65536) {
    const uint32_t n = (uint32_t)(hi - a < 65536 ? hi - a : 65536);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base + a), "r"(n)
                 : "memory");
  }
}

// Geometry of segment `seg` of `file`.
__device__ __forceinline__ SegGeom seg_geom(const Geom &g, const DevParams &p,
                                            uint32_t file, uint32_t seg) {
  SegGeom gm;
  gm.seg = seg;
  gm.n_f = file_size(g, file);
  gm.gbase = file_start(g, file);
  gm.p_s = (uint64_t)seg * g.L;
  gm.q_s = min(gm.p_s + g.L, gm.n_f);
  const uint64_t w1 = min(gm.q_s + p.mx, gm.n_f);
  // Window base: 32 bytes before the item, rounded down so that its global
  // byte index is 16-aligned.
  int64_t gb = (int64_t)(gm.gbase + gm.p_s) - 32;
  gb = gb >= 0 ? (gb & ~(int64_t)15) : -(((-gb) + 15) & ~(int64_t)15);
  gm.B = gb - (int64_t)gm.gbase;
  gm.W = (uint32_t)(((int64_t)w1 - gm.B + 31) >> 5);
  return gm;
}

__device__ __forceinline__ Bits bits_of(const MapSmem &m, uint32_t W) {
  return Bits{m.E, m.O, m.nz, m.sbO, m.locO, W};
}

// T bits (bits 16..31) of the 16 positions of v, whose first byte's
// predecessor is taken as equal to it (bit 16 is then 0; callers use only the
// top SeqLength-2 bits).
__device__ __forceinline__ uint32_t classify16_T(uint4 v, uint32_t mode) {
  uint32_t g0, l0, g1, l1, g2, l2, g3, l3;
  cmp_word(v.x, (v.x << 8) | (v.x & 0xffu), g0, l0);
  cmp_word(v.y, __funnelshift_l(v.x, v.y, 8), g1, l1);
  cmp_word(v.z, __funnelshift_l(v.y, v.z, 8), g2, l2);
  cmp_word(v.w, __funnelshift_l(v.z, v.w, 8), g3, l3);
  const uint32_t up = gather8(g0, g1) | (gather8(g2, g3) << 8);
  const uint32_t dn = gather8(l0, l1) | (gather8(l2, l3) << 8);
  return (mode == 0 ? up : dn) << 16;
}

// The natural cuts an item tabulates: run ends e in [lo, hi) give cut e + 1
// at index first + (rank of e among the E bits from lo on); those with e < eh
// are entries.  With want == false nothing is tabulated (repair pass).
struct CandRange {
  uint32_t lo, hi, eh, first, cap, ps_rel;
  bool want;
};

struct CandCount {
  uint32_t nc_nat;    // natural cuts in the range
  uint32_t nent_nat;  // of which entries
  uint32_t elo;       // E bits before lo
};

// E bits before rel position x (x <= 32 W), once sbE holds block-wide
// counts: the step's base plus a warp-wide count over the words of x's step
// before x.  Called by all lanes of a warp; each lane gets the result.
__device__ __forceinline__ uint32_t erank_warp(const MapSmem &m, uint32_t W, uint32_t etot,
                                               uint32_t x) {
  const uint32_t w = x >> 5;
  if (w >= W) return etot;
  const uint32_t lane = threadIdx.x & 31;
  uint32_t c = 0;
  for (uint32_t k = (w & ~63u) + lane; k <= w; k += 32) {
    uint32_t v = m.E[k];
    if (k == w) v &= (1u << (x & 31)) - 1u;
    c += __popc(v);
  }
  return m.sbE[w >> 6] + __reduce_add_sync(0xffffffffu, c);
}

// E and O bitmaps of the window [B, B + 32 W), their query tables and the
// item's natural cuts.  Warp k covers the words [k per, (k + 1) per) in steps
// of 64; per step, lane j takes words wb + j and wb + 32 + j (32 bytes each),
// so a ballot gives the nonzero-E mask in word order and one warp scan gives
// the O counts of both halves.  Three barriers: after the pass, after each
// warp has made its step counts block-wide, after the candidate scatter.
__device__ __forceinline__ CandCount seg_bitmaps(const SegGeom &gm, const Geom &g,
                                                 const DevParams &p, const MapSmem &m,
                                                 const CandRange &cr) {
  constexpr uint32_t kAll = 0xffffffffu;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const uint32_t W = gm.W;
  const uint8_t *base = g.data;
  const int64_t gwin = (int64_t)gm.gbase + gm.B;  // global byte index of rel 0
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
  uint32_t per = (W + nwarps - 1) / nwarps;
  per = (per + 63) & ~63u;
  const uint32_t w0 = min(warp * per, W);
  const uint32_t w1 = min(w0 + per, W);
  uint32_t carry_byte = 0, carry_T = 0;
  if (w0 < w1 && w0 > 0) {
    // T bits of the 16 positions before this warp's first word (only the top
    // SeqLength-2 of them matter, so the unknown byte before them is moot).
    const uint4 pv = load16(base, gwin + 32 * (int64_t)w0 - 16, g.total);
    carry_T = classify16_T(pv, p.mode);  // top 16 bits: the 16 positions before this word
    carry_byte = pv.w >> 24;
  }
  uint32_t cE = 0, cO = 0;  // E and O bits so far in this warp's words
  for (uint32_t wb = w0; wb < w1; wb += 64) {
    const uint32_t wa = wb + lane, wc = wa + 32;
    const bool la = wa < w1, lc = wc < w1;
    const int64_t gs = gwin + 32 * (int64_t)wb;
    uint4 a0, a1, c0, c1;
    if (gs >= 0 && (uint64_t)gs + 2048 <= g.total) {
      const uint4 *q = reinterpret_cast<const uint4 *>(base + gs) + 2 * lane;
      a0 = __ldg(q);
      a1 = __ldg(q + 1);
      c0 = __ldg(q + 64);
      c1 = __ldg(q + 65);
    } else {
      const int64_t ga = gs + 32 * lane, gc = ga + 1024;
      a0 = load16(base, ga, g.total);
      a1 = load16(base, ga + 16, g.total);
      c0 = load16(base, gc, g.total);
      c1 = load16(base, gc + 16, g.total);
    }
    const uint32_t lastA = a1.w >> 24, lastC = c1.w >> 24;
    uint32_t pbA = __shfl_up_sync(kAll, lastA, 1);
    uint32_t pbC = __shfl_up_sync(kAll, lastC, 1);
    const uint32_t lastA31 = __shfl_sync(kAll, lastA, 31);
    if (lane == 0) {
      pbA = carry_byte;
      pbC = lastA31;
    }
    uint32_t TA, OA, TC, OC;
    classify32(a0, a1, pbA, p.mode, TA, OA);
    classify32(c0, c1, pbC, p.mode, TC, OC);
    uint32_t ptA = __shfl_up_sync(kAll, TA, 1);
    uint32_t ptC = __shfl_up_sync(kAll, TC, 1);
    const uint32_t TA31 = __shfl_sync(kAll, TA, 31);
    if (lane == 0) {
      ptA = carry_T;
      ptC = TA31;
    }
    uint32_t EA = run_ends(ptA, TA, p.R), EC = run_ends(ptC, TC, p.R);
    if (!la) { EA = 0; OA = 0; }
    if (!lc) { EC = 0; OC = 0; }
    carry_byte = __shfl_sync(kAll, lastC, 31);
    carry_T = __shfl_sync(kAll, TC, 31);
    if (la) { m.E[wa] = EA; m.O[wa] = OA; }
    if (lc) { m.E[wc] = EC; m.O[wc] = OC; }
    const uint32_t nzA = __ballot_sync(kAll, EA != 0);
    const uint32_t nzC = __ballot_sync(kAll, EC != 0);
    const uint32_t stepE = __reduce_add_sync(kAll, __popc(EA) + __popc(EC));
    // O counts before each word within the step: first half in the low 16
    // bits, second half in the high 16 bits (each at most 1024).
    const uint32_t xv = __popc(OA) | (__popc(OC) << 16);
    uint32_t sv = xv;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(kAll, sv, d);
      if (lane >= d) sv += y;
    }
    const uint32_t tv = __shfl_sync(kAll, sv, 31);
    const uint32_t ev = sv - xv;
    const uint32_t tA = tv & 0xffffu;
    if (la) m.locO[wa] = (uint16_t)(ev & 0xffffu);
    if (lc) m.locO[wc] = (uint16_t)(tA + (ev >> 16));
    if (lane == 0) {
      m.nz[wb >> 5] = nzA;
      m.nz[(wb >> 5) + 1] = nzC;
      m.sbE[wb >> 6] = cE;
      m.sbO[wb >> 6] = cO;
    }
    cE += stepE;
    cO += tA + (tv >> 16);
  }
  if (lane == 0) {
    m.bscratch[warp] = cE;
    m.bscratch[32 + warp] = cO;
  }
  __syncthreads();

  // Warp bases (exclusive scans over the warps' totals) added to the step
  // counts of this warp's words.
  const uint32_t vE = lane < nwarps ? m.bscratch[lane] : 0u;
  const uint32_t vO = lane < nwarps ? m.bscratch[32 + lane] : 0u;
  uint32_t sE = vE, sO = vO;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t yE = __shfl_up_sync(kAll, sE, d);
    const uint32_t yO = __shfl_up_sync(kAll, sO, d);
    if (lane >= d) { sE += yE; sO += yO; }
  }
  const uint32_t etot = __shfl_sync(kAll, sE, 31);
  const uint32_t baseE = __shfl_sync(kAll, sE - vE, warp);
  const uint32_t baseO = __shfl_sync(kAll, sO - vO, warp);
  if (w0 < w1 && (baseE | baseO)) {  // a warp without words owns no step
    for (uint32_t st = (w0 >> 6) + lane; (st << 6) < w1; st += 32) {
      m.sbE[st] += baseE;
      m.sbO[st] += baseO;
    }
  }
  __syncthreads();

  CandCount cc;
  cc.elo = erank_warp(m, W, etot, cr.lo);
  cc.nc_nat = erank_warp(m, W, etot, cr.hi) - cc.elo;
  cc.nent_nat = erank_warp(m, W, etot, min(max(cr.eh, cr.lo), cr.hi)) - cc.elo;
  if (cr.want && cr.first + cc.nc_nat <= cr.cap) {
    // Steps that meet [lo, hi), one per warp: a warp scan gives the run ends
    // of the step before each word; in-range ones go to cpos by rank, and
    // erank_c gets the index of each word's first in-range run end.
    const uint32_t wlo = cr.lo >> 5, whi = (cr.hi + 31) >> 5;
    for (uint32_t st = (wlo >> 6) + warp; (st << 6) < whi; st += nwarps) {
      const uint32_t wb = st << 6;
      const uint32_t wa = wb + lane, wc = wa + 32;
      const uint32_t EA = wa < W ? m.E[wa] : 0u, EC = wc < W ? m.E[wc] : 0u;
      const uint32_t xv = __popc(EA) | (__popc(EC) << 16);
      uint32_t sv = xv;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kAll, sv, d);
        if (lane >= d) sv += y;
      }
      const uint32_t tA = __shfl_sync(kAll, sv, 31) & 0xffffu;
      const uint32_t ev = sv - xv;
      const uint32_t rbase = cr.first + m.sbE[st] - cc.elo;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t w = h ? wc : wa;
        if (w < wlo || w >= whi) continue;
        const uint32_t ew = h ? EC : EA;
        const uint32_t r0 = rbase + (h ? tA + (ev >> 16) : (ev & 0xffffu));
        const uint32_t bw = w << 5;
        uint32_t v = ew;
        uint32_t below_lo = 0;
        if (cr.lo > bw) {
          const uint32_t lmask = (1u << (cr.lo - bw)) - 1u;
          below_lo = __popc(ew & lmask);
          v &= ~lmask;
        }
        if (cr.hi - bw < 32) v &= (1u << (cr.hi - bw)) - 1u;
        m.erank_c[w - wlo] = (uint16_t)(r0 + below_lo);
        if (v) {
          uint32_t b = __ffs(v) - 1;
          uint32_t idx = r0 + __popc(ew & ((1u << b) - 1u));
          m.cpos[idx] = bw + b + 1;
          v &= v - 1;
          while (v) {  // words with two or more run ends are the rare case
            b = __ffs(v) - 1;
            v &= v - 1;
            m.cpos[++idx] = bw + b + 1;
          }
        }
      }
    }
    if (tid == 0 && cr.first) m.cpos[0] = cr.ps_rel;
  }
  __syncthreads();
  return cc;
}

// ---------------------------------------------------------------------------
// Map kernel: one block per item, no inter-block waits.
//   candidates  every natural cut x = e + 1 (E[e] set) with p_s <= x < q_s,
//               plus the file start for the first item of a file;
//   next        the chunker's next cut from each candidate, as the index of
//               that candidate, or a terminal code (first cut >= q_s) or an
//               escape code (a forced cut inside the item: not a candidate);
//   exits       the terminal of every entry candidate (those below
//               p_s + max_size), by following its chain of next codes, and
//               their distinct values.
// ---------------------------------------------------------------------------
// Instantiated per block size, each capped at 40 registers so that the
// blocks that shared memory allows (six of 256 threads at 64 KiB segments)
// are not limited by registers.
template <int kThreads, int kMinBlocks>
__global__ void __launch_bounds__(kThreads, kMinBlocks)
map_kernel(Geom g, DevParams p, WsPtrs ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t kMaxCand = g.cap;
  __shared__ SegShared sh;
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const uint32_t item = blockIdx.x;
  const uint32_t nitems = ws.hdr->nitems;
  if (item >= nitems) return;
  // Every warp finds the item's file and geometry itself: no barrier before
  // the bitmap pass.
  const uint32_t f = find_file_warp(ws.seg_base, g.nfiles, item);
  const SegGeom gm = seg_geom(g, p, f, item - ws.seg_base[f]);
  if (tid < 32 && !g.host) {
    const int64_t gwin = (int64_t)gm.gbase + gm.B;
    prefetch_l2(g.data, gwin, gwin + 32 * (int64_t)gm.W, g.total);
  }
  if (tid == 0) {
    ws.item_file[item] = f;
    sh.nc = 0;
    sh.nent = 0;
    sh.ninvalid = 0;
    sh.nimg = 0;
    sh.qhead = 0;
  }
  const MapSmem m = carve(smem_raw, gm.W, g.L);
  const int64_t B = gm.B;
  const uint64_t p_s = gm.p_s, n_f = gm.n_f;
  const uint32_t end_rel = end_rel_of(n_f, B);
  const uint32_t q_rel = (uint32_t)((int64_t)gm.q_s - B);
  const uint32_t ps_rel = (uint32_t)((int64_t)p_s - B);
  const uint32_t first = gm.seg == 0 ? 1u : 0u;
  // Candidate run ends e in [lo, hi): x = e + 1 in [p_s, q_s).  In a file's
  // first item, run ends before byte SeqLength-1 would need bytes before the
  // file start, so they are not candidates.  Entries: x < p_s + max_size.
  const uint32_t lo = first ? ps_rel + p.R - 1 : ps_rel - 1;
  const uint32_t hi = max(q_rel - 1, lo);
  const uint32_t ent_end = (uint32_t)((int64_t)min(p_s + (uint64_t)p.mx, n_f) - B);
  const CandRange cr{lo, hi, ent_end - 1, first, (uint32_t)kMaxCand, ps_rel, true};
  const CandCount cc = seg_bitmaps(gm, g, p, m, cr);
  const uint32_t nc = cc.nc_nat + first;
  const bool abnormal = nc > (uint32_t)kMaxCand;
  if (!abnormal && tid == 0) {
    sh.nc = nc;
    sh.nent = first ? 1u : cc.nent_nat;
  }
  __syncthreads();
  if (abnormal) {
    if (tid == 0) {
      ws.cand_n[item] = kAbnormal;
      ws.img_n[item] = 0;
      ws.state[item] = F_NOIMG;
      atomicAdd(&ws.hdr->stats[ST_ABNORMAL], 1u);
    }
    return;
  }

  // Next cut of every candidate, as a candidate index or a terminal code.
  // Lanes advance one scan region per iteration and take a new candidate
  // from a block-wide queue when theirs is done, so a warp's lanes stay busy
  // however many regions a chunk needs.
  const Bits bits = bits_of(m, gm.W);
  const uint32_t skip_min = p.mn > p.R ? p.mn - p.R : 0u;
  const int lane = tid & 31;
  for (int j = tid; j < kImgHash; j += nthreads) m.ihash[j] = kEscape;
  const uint32_t Wm1 = gm.W - 1;
  const uint32_t wlo = lo >> 5, lo_keep = ~((1u << (lo & 31)) - 1u);
  // Only as many warps as give each lane about kCandPerLane candidates take
  // part: a lane then runs through several chunks, so fewer lanes idle in
  // the tail of the longest chunk; the other warps wait at the barrier
  // without issuing.
  const uint32_t step_warps =
      min((uint32_t)(nthreads >> 5), max(1u, (nc + 32 * kCandPerLane - 1) / (32 * kCandPerLane)));
  uint32_t k = kNone, lim = 0, i = 0;
  bool more = (uint32_t)(tid >> 5) < step_warps;  // the queue may hold candidates
  while ((uint32_t)(tid >> 5) < step_warps) {
    if (more) {
      const uint32_t want = __ballot_sync(0xffffffffu, k == kNone);
      if (want) {
        const int leader = __ffs(want) - 1;
        uint32_t qb = 0;
        if (lane == leader) qb = atomicAdd(&sh.qhead, (uint32_t)__popc(want));
        qb = __shfl_sync(0xffffffffu, qb, leader);
        const uint32_t kk = qb + __popc(want & ((1u << lane) - 1u));
        if (k == kNone && kk < nc) {
          k = kk;
          const uint32_t c = m.cpos[kk];
          lim = (end_rel - c > p.mx) ? c + p.mx : end_rel;
          i = c + skip_min;
        }
        more = qb + __popc(want) < nc;
      }
    }
    if (__ballot_sync(0xffffffffu, k != kNone) == 0) break;
    const uint32_t y = region_step(bits, p, i, k != kNone ? lim : 0u);
    // The next cut as a code: terminal (at or after q_s), the index of the
    // candidate it is (its rank among the run ends from lo on), or escape (a
    // forced cut inside the item, which is not a candidate).
    const uint32_t ye = y - 1;
    const uint32_t w = min(ye >> 5, Wm1);
    const uint32_t ew = m.E[w];
    const uint32_t bit = 1u << (ye & 31);
    uint32_t code = kEscape;
    if (y >= q_rel) code = kTerminal | (y - ps_rel);
    else if (ye >= lo && ye < hi && (ew & bit))  // also keeps lanes without a cut in range
      code = m.erank_c[w - wlo] + __popc(ew & (bit - 1u) & (w == wlo ? lo_keep : ~0u));
    if (k != kNone && y != kNone) {
      // A candidate's next cut lies after it: a candidate code must be a
      // later index (anything else would be a table fault; escaping sends the
      // item to the exact repair pass).
      if (!(code & kTerminal) && (code <= k || code >= nc)) code = kEscape;
      m.cnxt[k] = code;
      k = kNone;
    }
  }
  __syncthreads();
  // Publish the candidate graph and every entry's exit; collect distinct exits.
  const uint32_t nent = sh.nent;
  uint32_t *gpos = ws.cand_pos + (uint64_t)item * kMaxCand;
  uint32_t *gnxt = ws.cand_nxt + (uint64_t)item * kMaxCand;
  uint32_t *gterm = ws.ent_term + (uint64_t)item * kMaxCand;
  for (uint32_t k = tid; k < nc; k += nthreads) {
    gpos[k] = m.cpos[k] - ps_rel;
    gnxt[k] = m.cnxt[k];
    if (k < nent) {
      // The entry's exit: follow its chain (indices only grow) to the code
      // that ends it.
      uint32_t t = m.cnxt[k];
      for (uint32_t hop = 0; !(t & kTerminal); ++hop) {
        t = hop < nc ? m.cnxt[t] : kEscape;  // indices grow: at most nc hops
      }
      const uint32_t ex = (t == kEscape) ? kEscape : (t & ~kTerminal);
      gterm[k] = ex;
      if (ex == kEscape) {
        atomicAdd(&sh.ninvalid, 1u);
      } else {
        uint32_t slot = (ex * 2654435761u) >> (32 - 7);  // kImgHash = 128
        for (int probe = 0; probe < kImgHash; ++probe) {
          const uint32_t prev = atomicCAS(&m.ihash[slot], kEscape, ex);
          if (prev == kEscape) { atomicAdd(&sh.nimg, 1u); break; }
          if (prev == ex) break;
          slot = (slot + 1) & (kImgHash - 1);
        }
      }
    }
  }
  __syncthreads();
  const bool img_ok = sh.ninvalid == 0 && sh.nimg <= (uint32_t)kMaxImage;
  if (tid == 0) sh.nimg = 0;
  __syncthreads();
  if (img_ok) {
    for (int i = tid; i < kImgHash; i += nthreads) {
      const uint32_t ex = m.ihash[i];
      if (ex != kEscape) {
        const uint32_t at = atomicAdd(&sh.nimg, 1u);
        ws.img[(uint64_t)item * kMaxImage + at] = p_s + ex;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    ws.cand_n[item] = nc;
    ws.ent_n[item] = nent;
    ws.img_n[item] = img_ok ? sh.nimg : 0u;
    ws.state[item] = img_ok ? F_IMG : F_NOIMG;
    if (!img_ok) atomicAdd(&ws.hdr->stats[ST_NOIMG], 1u);
  }
}

// ---------------------------------------------------------------------------
// Resolve kernel: one warp per item, items taken in ticket order so that
// every item's predecessors are running or done.
// ---------------------------------------------------------------------------
struct ResShared {
  uint32_t item, file, seg, first_item, nc, nent;
  uint64_t p_s, q_s;
};

// Index of the entry at y (file-relative) among the item's tabulated
// entries (positions staged in shared memory), or -1.
__device__ __forceinline__ int entry_index(const ResShared &r, const uint32_t *spos,
                                           uint64_t y) {
  if (r.nc == kAbnormal || y < r.p_s || y >= r.q_s) return -1;
  const uint32_t want = (uint32_t)(y - r.p_s);
  uint32_t lo = 0, hi = r.nent;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint32_t v = spos[mid];
    if (v == want) return (int)mid;
    if (v < want) lo = mid + 1; else hi = mid;
  }
  return -1;
}

// Exit of `item` from entry position y (file-relative), from its table; kBad
// when y is not a tabulated entry or its chain escapes.  One lane.
__device__ uint64_t exit_of(const WsPtrs &ws, const ResShared &r, const uint32_t *spos,
                           uint64_t y, uint32_t kMaxCand) {
  if (y >= r.q_s) return y;
  const int k = entry_index(r, spos, y);
  if (k < 0) return kBad;
  const uint32_t t = ws.ent_term[(uint64_t)r.item * kMaxCand + k];
  return t == kEscape ? kBad : r.p_s + t;
}

// True entry by decoupled look-back (one warp).  Going back from item-1, each
// predecessor k either has published its true exit (stop), or its map from
// the image of k-1 to its exits (compose and continue), or no map (wait for
// its true exit).  The composite is one value per lane: lane j holds the exit
// of item-1 reached from value j of the current image.  A composite that is
// the same for every value settles the entry at once.
__device__ uint64_t lookback(const ResShared &r, const WsPtrs &ws, uint64_t limit_ns) {
  const int lane = threadIdx.x & 31;
  const uint32_t item = r.item;
  uint32_t k = item - 1;
  uint64_t comp = 0;
  bool have = false, started = false, waited = false;
  uint32_t steps = 0;
  uint64_t x = kBad;
  while (true) {
    // Lane 0 waits; every lane acquires for its own reads but all branch on
    // lane 0's snapshot (flags only gain bits).
    uint32_t st = 0;
    if (lane == 0) st = wait_any(&ws.state[k], F_INCL | F_AGG | F_NOAGG, ws.hdr, limit_ns);
    st = __shfl_sync(0xffffffffu, st, 0);
    if (st == 0) break;  // timed out; status is recorded
    (void)ld_acquire(&ws.state[k]);
    __syncwarp();
    if (!(st & F_INCL) && (st & F_NOAGG)) {
      if (lane == 0) st = wait_any(&ws.state[k], F_INCL, ws.hdr, limit_ns);
      st = __shfl_sync(0xffffffffu, st, 0);
      waited = true;
      if (st == 0) break;
      (void)ld_acquire(&ws.state[k]);
      __syncwarp();
    }
    if (st & F_INCL) {
      const uint64_t e = __ldcg(&ws.incl[k]);  // true exit of k = entry of k+1
      if (!started || e == kBad) { x = e; break; }
      const uint32_t n = __ldcg(&ws.img_n[k]);
      const uint64_t v = (lane < (int)n) ? __ldcg(&ws.img[(uint64_t)k * kMaxImage + lane]) : kBad;
      const uint32_t hit = __ballot_sync(0xffffffffu, lane < (int)n && v == e && have);
      if (hit) { x = __shfl_sync(0xffffffffu, comp, __ffs(hit) - 1); break; }
      // Outside the composite's domain: wait for item-1's own true exit.
      if (lane == 0) st = wait_any(&ws.state[item - 1], F_INCL, ws.hdr, limit_ns);
      st = __shfl_sync(0xffffffffu, st, 0);
      waited = true;
      if (st) {
        (void)ld_acquire(&ws.state[item - 1]);
        __syncwarp();
        x = __ldcg(&ws.incl[item - 1]);
      }
      break;
    }
    // F_AGG: map from the image of k-1 to the exits of k.
    const uint32_t n_agg = __ldcg(&ws.img_n[k - 1]);
    const uint64_t av = (lane < (int)n_agg) ? __ldcg(&ws.agg[(uint64_t)k * kMaxImage + lane]) : kBad;
    if (!started) {
      comp = av;
      have = lane < (int)n_agg && av != kBad;
      started = true;
    } else {
      const uint32_t n_img = __ldcg(&ws.img_n[k]);
      const uint64_t im = (lane < (int)n_img) ? __ldcg(&ws.img[(uint64_t)k * kMaxImage + lane]) : kBad;
      uint64_t nc = 0;
      bool nh = false;
      for (uint32_t j = 0; j < n_img; ++j) {
        const uint64_t imj = __shfl_sync(0xffffffffu, im, j);
        const uint64_t cj = __shfl_sync(0xffffffffu, comp, j);
        const bool hj = __shfl_sync(0xffffffffu, have, j);
        if (!nh && lane < (int)n_agg && av != kBad && av == imj && hj) { nc = cj; nh = true; }
      }
      comp = nc;
      have = nh;
    }
    ++steps;
    const uint32_t hv = __ballot_sync(0xffffffffu, have);
    if (hv == 0) {  // nothing composes any more: wait for item-1's true exit
      if (lane == 0) st = wait_any(&ws.state[item - 1], F_INCL, ws.hdr, limit_ns);
      st = __shfl_sync(0xffffffffu, st, 0);
      waited = true;
      if (st) {
        (void)ld_acquire(&ws.state[item - 1]);
        __syncwarp();
        x = __ldcg(&ws.incl[item - 1]);
      }
      break;
    }
    const uint64_t c0 = __shfl_sync(0xffffffffu, comp, __ffs(hv) - 1);
    if (__all_sync(0xffffffffu, !have || comp == c0)) { x = c0; break; }
    --k;  // k > first item: the first item publishes F_INCL, never F_AGG
  }
  if (lane == 0) {
    atomicAdd(&ws.hdr->stats[ST_LB_STEPS], steps);
    if (waited) atomicAdd(&ws.hdr->stats[ST_LB_WAITS], 1u);
  }
  return x;
}

// Each warp of a block resolves its own item (blocks hold up to
// kResolveWarps warps so that more items are in flight per SM).
constexpr int kResolveWarps = 4;

__global__ void __launch_bounds__(32 * kResolveWarps)
resolve_kernel(Geom g, WsPtrs ws) {
  __shared__ ResShared rs[kResolveWarps];
  // The item's candidate positions and links, staged by the warp with
  // coalesced loads: entry lookups and the walk along the links then read
  // shared memory instead of one dependent global load per cut.
  extern __shared__ uint32_t rstage[];  // per warp: [cap] positions, [cap] links
  const uint32_t kMaxCand = g.cap;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  ResShared &r = rs[wid];
  uint32_t tk = 0;
  if (lane == 0) tk = atomicAdd(&ws.hdr->ticket, 1u);
  tk = __shfl_sync(0xffffffffu, tk, 0);
  const uint32_t fw = (tk < ws.hdr->nitems) ? find_file_warp(ws.seg_base, g.nfiles, tk) : 0u;
  if (lane == 0) {
    const uint32_t item = tk;
    r.item = item;
    if (item < ws.hdr->nitems) {
      const uint32_t f = fw;
      r.file = f;
      r.first_item = ws.seg_base[f];
      r.seg = item - r.first_item;
      r.p_s = (uint64_t)r.seg * g.L;
      r.q_s = min(r.p_s + g.L, file_size(g, f));
      r.nc = ws.cand_n[item];
      r.nent = ws.ent_n[item];
    }
  }
  __syncwarp();
  const uint32_t item = r.item;
  if (item >= ws.hdr->nitems) return;
  uint32_t *spos = rstage + (size_t)wid * 2 * kMaxCand, *snxt = spos + kMaxCand;
  {
    const uint32_t ncs = r.nc == kAbnormal ? 0u : r.nc;
    const uint32_t *gpos = ws.cand_pos + (uint64_t)item * kMaxCand;
    const uint32_t *gnxt = ws.cand_nxt + (uint64_t)item * kMaxCand;
    for (uint32_t j = lane; j < ncs; j += 32) {
      spos[j] = __ldcg(gpos + j);
      snxt[j] = __ldcg(gnxt + j);
    }
    __syncwarp();
  }
  uint64_t x = 0;
  if (r.seg > 0) {
    // The map from the predecessor's image to this item's exits.
    const uint32_t pst = ws.state[item - 1];  // written by the map kernel
    const bool ok = (pst & F_IMG) != 0;
    const uint32_t n = ok ? ws.img_n[item - 1] : 0u;
    if (lane < (int)n) {
      const uint64_t y = ws.img[(uint64_t)(item - 1) * kMaxImage + lane];
      ws.agg[(uint64_t)item * kMaxImage + lane] = exit_of(ws, r, spos, y, g.cap);
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      atomicOr(&ws.state[item], ok ? F_AGG : F_NOAGG);
    }
    x = lookback(r, ws, g.wait_ns);
  }
  // Emission from x along the candidate links (lane 0).  When x is not known
  // or is not one of the item's tabulated entries (a forced cut entered it),
  // the item's first entry is taken instead: its cuts and exit let the items
  // after it resolve, and since the recorded entry is then not the
  // predecessor's exit, the verify pass sends the item to the repair pass.
  if (lane == 0) {
    uint64_t *out = ws.slot + (uint64_t)item * ws.slot_cap;
    uint32_t nout = 0;
    uint64_t exit_pos = kBad, entry = x;
    bool done = false;
    if (x != kBad && x >= r.q_s) {
      exit_pos = x;  // the entry lies past the item: no cut inside it
      done = true;
    } else if (r.nc != kAbnormal) {
      int k = x != kBad ? entry_index(r, spos, x) : -1;
      const bool guess = k < 0 && r.nent > 0;
      if (guess) {
        k = 0;
        entry = r.p_s + spos[0];
      }
      if (k >= 0) {
        uint32_t code = snxt[k];
        while (!(code & kTerminal) && nout < ws.slot_cap) {
          if (code >= r.nc) { code = kEscape; break; }  // never: codes are checked when made
          out[nout++] = r.p_s + spos[code];
          code = snxt[code];
        }
        if (code != kEscape && nout < ws.slot_cap) {
          exit_pos = r.p_s + (code & ~kTerminal);
          out[nout++] = exit_pos;
          done = true;
        }
      }
      if (guess && done) atomicAdd(&ws.hdr->stats[ST_REPLAYED], 1u);
    }
    if (!done) {
      nout = 0;
      exit_pos = kBad;
      entry = x;
      atomicAdd(&ws.hdr->stats[ST_REPLAYED], 1u);
    }
    ws.count[item] = nout;
    ws.incl[item] = exit_pos;
    ws.entry[item] = entry;
    __threadfence();
    atomicOr(&ws.state[item], F_INCL);
    atomicAdd(&ws.hdr->stats[ST_ITEMS], 1u);
  }
}

// Verify: item s of a file is consistent when it was emitted and its entry
// equals the exit its predecessor computed.  By induction from the file start
// (always a true entry), a file whose items are all consistent is exact.
__device__ __forceinline__ bool item_consistent(const WsPtrs &ws, uint64_t i, uint32_t s) {
  bool ok = (ws.state[i] & F_INCL) && ws.incl[i] != kBad && ws.entry[i] != kBad;
  if (ok) ok = ws.entry[i] == (s > 0 ? ws.incl[i - 1] : 0ull);
  return ok;
}

// Rounds 0 .. kRepairRounds-1 list the first item of every run of
// inconsistent items (and flag it) for the parallel repair; the last round
// records the first inconsistent item of each file for the sequential repair.
__global__ void verify_kernel(Geom g, WsPtrs ws, uint32_t round) {
  // Nothing was inconsistent in the previous round, so nothing changed.
  if (round > 0 && ws.hdr->nruns[round - 1] == 0) return;
  const uint32_t nitems = ws.hdr->nitems;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nitems;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t f = ws.item_file[i];
    const uint32_t s = (uint32_t)i - ws.seg_base[f];
    const bool ok = item_consistent(ws, i, s);
    if (round < kRepairRounds) {
      const bool start = !ok && (s == 0 || item_consistent(ws, i - 1, s - 1));
      if (start) {
        ws.runs[atomicAdd(&ws.hdr->nruns[round], 1u)] = (uint32_t)i;
        atomicOr(&ws.state[i], F_RUN);
      } else if (ws.state[i] & F_RUN) {
        atomicAnd(&ws.state[i], ~F_RUN);
      }
      if (round == 0 && !ok) atomicAdd(&ws.hdr->stats[ST_INCONSISTENT], 1u);
    } else if (!ok) {
      atomicMin(&ws.first_bad[f], s);
    }
  }
}

// Re-chunk `item` (segment `seg` of `file`) from entry `cur` (file-relative):
// the block rebuilds the bitmaps from the input, thread 0 steps the chunker.
// Called by every thread of the block; returns the item's new exit.
__device__ uint64_t rechunk_item(const Geom &g, const DevParams &p, const WsPtrs &ws,
                                 SegShared &sh, unsigned char *smem_raw, uint32_t item,
                                 uint32_t file, uint32_t seg, uint64_t cur) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    sh.gm = seg_geom(g, p, file, seg);
    atomicAdd(&ws.hdr->stats[ST_RECOMPUTED], 1u);
  }
  __syncthreads();
  const SegGeom gm = sh.gm;
  const MapSmem m = carve(smem_raw, gm.W, g.L);
  (void)seg_bitmaps(gm, g, p, m, CandRange{0, 0, 0, 0, 0, 0, false});
  if (tid == 0) {
    const Bits bits = bits_of(m, gm.W);
    const int64_t B = gm.B;
    const uint32_t end_rel = end_rel_of(gm.n_f, B);
    const uint32_t q_rel = (uint32_t)((int64_t)gm.q_s - B);
    uint64_t *out = ws.slot + (uint64_t)item * ws.slot_cap;
    uint32_t nout = 0;
    uint32_t c = (uint32_t)((int64_t)cur - B);
    while (c < q_rel && nout < ws.slot_cap) {
      c = chunk_step(bits, p, c, end_rel);
      out[nout++] = (uint64_t)(B + (int64_t)c);
    }
    const uint64_t e = nout ? (uint64_t)(B + (int64_t)c) : cur;
    ws.count[item] = nout;
    ws.entry[item] = cur;
    ws.incl[item] = e;
    atomicOr(&ws.state[item], F_INCL);
    sh.exit = e;
  }
  __syncthreads();
  const uint64_t e = sh.exit;
  __syncthreads();
  return e;
}

// Parallel repair: persistent blocks take runs from the list of this round.
// A run is re-chunked item by item from the exit of the item before it, until
// an item's recorded entry equals the new exit (it was already chunked from
// the right entry) or the next run's first item (which its own block takes).
// A run whose starting exit changes meanwhile is found by the next round.
__global__ void __launch_bounds__(512)
run_repair_kernel(Geom g, DevParams p, WsPtrs ws, uint32_t round) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SegShared sh;
  const int tid = threadIdx.x;
  const uint32_t nruns = ws.hdr->nruns[round];
  while (true) {
    if (tid == 0) sh.flag = atomicAdd(&ws.hdr->runq[round], 1u);
    __syncthreads();
    const uint32_t r = sh.flag;
    __syncthreads();
    if (r >= nruns) return;
    const uint32_t i0 = ws.runs[r];
    const uint32_t f = ws.item_file[i0];
    const uint32_t base = ws.seg_base[f], end = ws.seg_base[f + 1];
    uint64_t cur = (i0 == base) ? 0ull : __ldcg(&ws.incl[i0 - 1]);
    for (uint32_t it = i0; it < end; ++it) {
      if (it > i0) {
        if (tid == 0) {
          const uint32_t st = __ldcg(&ws.state[it]);
          sh.flag = (st & F_RUN) || ((st & F_INCL) && __ldcg(&ws.incl[it]) != kBad &&
                                     __ldcg(&ws.entry[it]) == cur);
        }
        __syncthreads();
        const bool stop = sh.flag != 0;
        __syncthreads();
        if (stop) break;
      }
      cur = rechunk_item(g, p, ws, sh, smem_raw, it, f, it - base, cur);
    }
  }
}

// Sequential repair (last resort): one block per file that is still
// inconsistent; from its first inconsistent item on, every item whose
// recorded entry is not its predecessor's exit is re-chunked.
__global__ void __launch_bounds__(512)
repair_kernel(Geom g, DevParams p, WsPtrs ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SegShared sh;
  const int tid = threadIdx.x;
  for (uint64_t f = blockIdx.x; f < g.nfiles; f += gridDim.x) {
    const uint32_t fb = ws.first_bad[f];
    if (fb == 0xffffffffu) continue;
    const uint32_t base = ws.seg_base[f];
    const uint32_t nseg = ws.seg_base[f + 1] - base;
    uint64_t cur = fb ? ws.incl[base + fb - 1] : 0;
    for (uint32_t s = fb; s < nseg; ++s) {
      const uint32_t item = base + s;
      if (tid == 0) {
        sh.flag = !((ws.state[item] & F_INCL) && ws.incl[item] != kBad &&
                    ws.entry[item] == cur);
      }
      __syncthreads();
      const bool run = sh.flag != 0;
      __syncthreads();
      if (run) cur = rechunk_item(g, p, ws, sh, smem_raw, item, (uint32_t)f, s, cur);
      else cur = __ldcg(&ws.incl[item]);
    }
  }
}

// ---------------------------------------------------------------------------
// Compaction: exclusive scan of per-item cut counts, copy to the CSR output.
// ---------------------------------------------------------------------------
__global__ void count_tiles_kernel(WsPtrs ws) {
  __shared__ uint32_t red[32];
  const uint32_t nitems = ws.hdr->nitems;
  const uint64_t i = (uint64_t)blockIdx.x * kItemTile + threadIdx.x;
  uint32_t v = (threadIdx.x < kItemTile && i < nitems) ? ws.count[i] : 0u;
  for (int d = 16; d; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    ws.itile[blockIdx.x] = s;
  }
}

// kEmitSplit blocks share each tile: every one scans the tile's counts and
// copies kItemTile / kEmitSplit of its items, so that a short stream (a
// tile or two) is not copied by one block.
__global__ void emit_kernel(Geom g, WsPtrs ws, uint64_t *d_cuts, uint64_t cap,
                            uint64_t *d_cut_offsets, uint64_t *d_count) {
  __shared__ uint32_t scratch[32];
  __shared__ uint64_t red64[32];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t offs[kItemTile + 1];
  const uint32_t nitems = ws.hdr->nitems;
  const uint32_t tile = blockIdx.x / kEmitSplit, sub = blockIdx.x % kEmitSplit;
  const uint64_t lo = (uint64_t)tile * kItemTile;
  uint64_t part = 0;
  for (uint64_t t = threadIdx.x; t < tile; t += blockDim.x) part += ws.itile[t];
  for (int d = 16; d; d >>= 1) part += __shfl_down_sync(0xffffffffu, part, d);
  if ((threadIdx.x & 31) == 0) red64[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red64[w];
    s_prefix = s;
  }
  __syncthreads();
  const uint64_t i = lo + threadIdx.x;
  const uint32_t c = (i < nitems) ? ws.count[i] : 0u;
  uint32_t tot;
  const uint32_t ex = block_excl_scan(c, scratch, &tot);
  offs[threadIdx.x] = ex;
  if (threadIdx.x == 0) offs[kItemTile] = tot;
  __syncthreads();
  const uint64_t prefix = s_prefix;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kPerSub = kItemTile / kEmitSplit;
  for (int it = sub * kPerSub + warp; it < (int)(sub + 1) * kPerSub; it += blockDim.x >> 5) {
    const uint64_t item = lo + it;
    if (item >= nitems) break;
    const uint32_t n = ws.count[item];
    const uint64_t at = prefix + offs[it];
    if (at + n > cap) {  // cannot happen for a correct cut list; never write past cap
      if (lane == 0) atomicExch(&ws.hdr->status, (uint32_t)SEQCDC_ECAPACITY);
      continue;
    }
    const uint64_t *src = ws.slot + item * ws.slot_cap;
    uint64_t *dst = d_cuts + at;
    for (uint32_t j = lane; j < n; j += 32) dst[j] = src[j];
  }
  // CSR offsets of the files whose first item index falls in [lo, lo+tile)
  // (by the tile's first block).
  const uint64_t hi = lo + kItemTile;
  if (sub == 0 && lo <= nitems) {
    uint64_t a = 0, b = g.nfiles + 1;  // lower_bound(seg_base, lo)
    while (a < b) {
      const uint64_t mid = (a + b) >> 1;
      if (ws.seg_base[mid] < lo) a = mid + 1; else b = mid;
    }
    for (uint64_t f = a + threadIdx.x; f <= g.nfiles; f += blockDim.x) {
      const uint32_t sb = ws.seg_base[f];
      if (sb >= hi) break;
      const uint64_t v = prefix + offs[sb - lo];
      if (d_cut_offsets) d_cut_offsets[f] = v;
      if (d_count && f == g.nfiles) *d_count = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool params_ok(const seqcdc_params_t *p) {
  if (!p) return false;
  if (p->mode > 1) return false;
  if (p->seq_length < 2 || p->seq_length > kMaxSeqLength) return false;
  if (p->min_size < 1 || p->max_size < p->min_size) return false;
  if (p->max_size > kMaxMaxSize) return false;
  return true;
}

uint32_t max_words(uint32_t L, uint64_t mx) {
  return (uint32_t)((L + mx + 64 + 31) / 32 + 2);
}

constexpr size_t kSmemBudget = 220 * 1024;

// Default segment: 64 KiB (at least max_size), with 256 threads: four
// blocks share an SM, which hides the latency of each block's barriers and
// of its longest chunk better than fewer, larger blocks.
uint32_t default_segment(uint64_t mx) { return mx > 65536u ? (uint32_t)mx : 65536u; }

uint32_t pick_segment(const seqcdc_params_t *p, const seqcdc_tuning_t *t) {
  uint32_t L = (t && t->segment_bytes) ? t->segment_bytes
                                       : default_segment(p ? p->max_size : 0);
  // An item must be at least max_size long so that its entries (natural cuts
  // below p_s + max_size) all lie inside it.
  if (p && L < p->max_size) L = (uint32_t)p->max_size;
  L = (L + 1023u) & ~1023u;
  if (L < 4096u) L = 4096u;
  if (L > (1u << 20)) L = 1u << 20;
  // Shrink until the block's shared memory fits (never below max_size).
  const uint64_t mx = p ? p->max_size : 0;
  while (L > 4096u && L - 1024u >= mx &&
         map_smem_bytes(max_words(L, mx), L) > kSmemBudget)
    L -= 1024u;
  return L;
}

// Which path a call takes: the tuning's choice, else the chain walk when
// the call has many chains to walk at once (each piece is a chain one warp
// walks): batches of many files, or at least SEQCDC_WALK_MIN_PIECES full
// pieces of input; the segment map otherwise (a short stream or a batch of
// few small files gives too few chains).
bool use_walk(const seqcdc_params_t *p, const seqcdc_tuning_t *t, uint64_t total,
              uint64_t nfiles, bool batch) {
  const uint32_t a = t ? t->algorithm : SEQCDC_ALGO_AUTO;
  if (a == SEQCDC_ALGO_WALK) return true;
  if (a == SEQCDC_ALGO_MAP) return false;
  if (batch && nfiles >= SEQCDC_WALK_MIN_FILES) return true;
  return total / seqcdc_walk::pick_piece(p, t) >= SEQCDC_WALK_MIN_PIECES;
}

size_t workspace_for(const seqcdc_params_t *p, uint64_t total, uint64_t nfiles,
                     const seqcdc_tuning_t *t, bool batch);

uint32_t pick_threads(const seqcdc_tuning_t *t) {
  uint32_t n = (t && t->block_threads) ? t->block_threads : 256u;
  if (n != 128u && n != 256u && n != 512u) n = 256u;
  return n;
}

Layout make_layout(const seqcdc_params_t *p, uint64_t total, uint64_t nfiles,
                   uint32_t L) {
  Layout l{};
  l.L = L;
  l.imax = (total + L - 1) / L + nfiles + 1;
  l.nftiles = (nfiles + kFileTile - 1) / kFileTile;
  if (l.nftiles == 0) l.nftiles = 1;
  l.nitiles = (l.imax + 1 + kItemTile - 1) / kItemTile;
  l.slot_cap = (uint32_t)((L + p->max_size) / p->min_size + 2);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  l.hdr = take(sizeof(WsHeader));
  l.seg_base = take((nfiles + 1) * 4);
  l.ftile = take(l.nftiles * 4);
  l.state = take(l.imax * 4);
  l.incl = take(l.imax * 8);
  l.entry = take(l.imax * 8);
  l.first_bad = take((nfiles + 1) * 4);
  l.count = take(l.imax * 4);
  l.img_n = take(l.imax * 4);
  l.img = take(l.imax * kMaxImage * 8);
  l.agg = take(l.imax * kMaxImage * 8);
  l.cand_n = take(l.imax * 4);
  l.ent_n = take(l.imax * 4);
  l.cand_pos = take(l.imax * (size_t)cand_cap(L) * 4);
  l.cand_nxt = take(l.imax * (size_t)cand_cap(L) * 4);
  l.ent_term = take(l.imax * (size_t)cand_cap(L) * 4);
  l.slot = take(l.imax * (size_t)l.slot_cap * 8);
  l.itile = take(l.nitiles * 4);
  l.runs = take(l.imax * 4);
  l.item_file = take(l.imax * 4);
  l.total = o;
  return l;
}

WsPtrs ws_ptrs(void *d_ws, const Layout &l) {
  char *b = static_cast<char *>(d_ws);
  WsPtrs w;
  w.hdr = reinterpret_cast<WsHeader *>(b + l.hdr);
  w.seg_base = reinterpret_cast<uint32_t *>(b + l.seg_base);
  w.ftile = reinterpret_cast<uint32_t *>(b + l.ftile);
  w.state = reinterpret_cast<uint32_t *>(b + l.state);
  w.incl = reinterpret_cast<uint64_t *>(b + l.incl);
  w.entry = reinterpret_cast<uint64_t *>(b + l.entry);
  w.first_bad = reinterpret_cast<uint32_t *>(b + l.first_bad);
  w.count = reinterpret_cast<uint32_t *>(b + l.count);
  w.img_n = reinterpret_cast<uint32_t *>(b + l.img_n);
  w.img = reinterpret_cast<uint64_t *>(b + l.img);
  w.agg = reinterpret_cast<uint64_t *>(b + l.agg);
  w.cand_n = reinterpret_cast<uint32_t *>(b + l.cand_n);
  w.ent_n = reinterpret_cast<uint32_t *>(b + l.ent_n);
  w.cand_pos = reinterpret_cast<uint32_t *>(b + l.cand_pos);
  w.cand_nxt = reinterpret_cast<uint32_t *>(b + l.cand_nxt);
  w.ent_term = reinterpret_cast<uint32_t *>(b + l.ent_term);
  w.slot = reinterpret_cast<uint64_t *>(b + l.slot);
  w.itile = reinterpret_cast<uint32_t *>(b + l.itile);
  w.runs = reinterpret_cast<uint32_t *>(b + l.runs);
  w.item_file = reinterpret_cast<uint32_t *>(b + l.item_file);
  w.slot_cap = l.slot_cap;
  return w;
}

size_t workspace_for(const seqcdc_params_t *p, uint64_t total, uint64_t nfiles,
                     const seqcdc_tuning_t *t, bool batch) {
  if (use_walk(p, t, total, nfiles, batch))
    return seqcdc_walk::workspace_bytes(p, total, nfiles, seqcdc_walk::pick_piece(p, t));
  return make_layout(p, total, nfiles, pick_segment(p, t)).total;
}

thread_local cudaEvent_t g_prof_begin = nullptr;
thread_local cudaEvent_t g_prof_end = nullptr;
thread_local uint64_t g_wait_ns = kWaitNs;

constexpr int kMaxDevices = 64;

// Streaming multiprocessors of the current device (cached per device); 0 on
// error.
int sm_count() {
  static std::mutex mu;
  static int n[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 0;
  std::lock_guard<std::mutex> lock(mu);
  if (!n[dev] && cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    n[dev] = 0;
  return n[dev];
}

// Allow `smem` bytes of dynamic shared memory for the map kernel of this
// block size and for the repair kernels on the current device; remembered per
// device so that the attribute is set once per size.
bool smem_configured(uint32_t threads, size_t smem,
                     void (*map_fn)(Geom, DevParams, WsPtrs)) {
  static std::mutex mu;
  static size_t done[kMaxDevices][3] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  const int k = threads == 128u ? 0 : threads == 512u ? 2 : 1;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev][k] >= smem) return true;
  if (cudaFuncSetAttribute(map_fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(repair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(run_repair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return false;
  done[dev][k] = smem;
  return true;
}

// The same for the resolve kernel's staging area (segments over 768 KiB).
bool resolve_smem_configured(size_t smem) {
  static std::mutex mu;
  static size_t done[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev] >= smem) return true;
  if (cudaFuncSetAttribute(resolve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess)
    return false;
  done[dev] = smem;
  return true;
}

// The path a call takes: use_walk's rule, and for AUTO with a workspace too
// small for the segment map but large enough for the chain walk, the walk
// (same output): a workspace sized for a larger batch then serves every
// smaller call, as the walk's workspace grows with the bytes and the files
// while the map's is larger.
bool decide_walk(const seqcdc_params_t *p, uint64_t total, uint64_t nfiles, bool batch,
                 size_t ws_bytes, const seqcdc_tuning_t *tuning) {
  bool walk = use_walk(p, tuning, total, nfiles, batch);
  if (!walk && (!tuning || tuning->algorithm == SEQCDC_ALGO_AUTO) &&
      ws_bytes < make_layout(p, total, nfiles, pick_segment(p, tuning)).total &&
      ws_bytes >= seqcdc_walk::workspace_bytes(p, total, nfiles,
                                               seqcdc_walk::pick_piece(p, tuning)))
    walk = true;
  return walk;
}

// Where the input of a call lives.  Device (or managed) memory: 0.  Pinned
// host memory mapped into the device's address space: 1, with *dev set to
// the address the device reads it at (the kernels read it in place).
// Pageable host memory, which the device cannot read: -1.
int data_kind(const uint8_t *ptr, const uint8_t **dev) {
  *dev = ptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();  // not a CUDA pointer: treated as device memory
    return 0;
  }
  if (a.type == cudaMemoryTypeUnregistered) return -1;
  if (a.type != cudaMemoryTypeHost) return 0;
  if (!a.devicePointer) return -1;  // pinned but not mapped
  *dev = static_cast<const uint8_t *>(a.devicePointer);
  return 1;
}

int run(const seqcdc_params_t *p, const uint8_t *d_data, uint64_t total,
        const uint64_t *d_offsets, uint64_t nfiles, uint64_t *d_cuts,
        uint64_t cap, uint64_t *d_cut_offsets, uint64_t *d_count, void *d_ws,
        size_t ws_bytes, const seqcdc_tuning_t *tuning, void *stream,
        bool locate = false) {
  if (!params_ok(p)) return SEQCDC_EINVAL;
  if (!d_ws || ((uintptr_t)d_ws & 255u)) return SEQCDC_EINVAL;
  if (total > 0 && (!d_data || ((uintptr_t)d_data & 15u))) return SEQCDC_EINVAL;
  if (total > 0 && !d_cuts) return SEQCDC_EINVAL;
  // With `locate`, where the input lives decides how it is read; input the
  // device cannot read is refused after the size checks, before any launch.
  const int kind = locate && total > 0 ? data_kind(d_data, &d_data) : 0;
  const bool host_data = kind == 1;
  bool walk = decide_walk(p, total, nfiles, d_offsets != nullptr, ws_bytes, tuning);
  // Input read in place from host memory: AUTO takes the chain walk, which
  // reads only the windows its scan reaches, when the workspace allows it.
  if (host_data && !walk && (!tuning || tuning->algorithm == SEQCDC_ALGO_AUTO) &&
      ws_bytes >= seqcdc_walk::workspace_bytes(p, total, nfiles,
                                               seqcdc_walk::pick_piece(p, tuning)))
    walk = true;
  if (walk) {
    if (cap < total / p->min_size + nfiles) return SEQCDC_ECAPACITY;
    uint32_t piece = seqcdc_walk::pick_piece(p, tuning);
    if (ws_bytes < seqcdc_walk::workspace_bytes(p, total, nfiles, piece))
      return SEQCDC_ECAPACITY;
    // Host-resident input with chains to spare (at least 4,096 pieces of
    // twice the default): twice the default piece, so fewer junction walks
    // re-read bytes across the host link (10,000-file batch: 4.16 ms against
    // 4.38 ms); a 1 GiB stream keeps the default (1.44 ms against 1.85 ms:
    // its chains, not its bytes, bound it).  Larger pieces need less
    // workspace.
    if (host_data && !(tuning && tuning->piece_bytes) && total / (2ull * piece) >= 4096u)
      piece = piece > (32u << 20) ? (64u << 20) : 2u * piece;
    if (kind < 0) return SEQCDC_EINVAL;
    const int sms_w = sm_count();
    if (sms_w <= 0) return SEQCDC_ECUDA;
    return seqcdc_walk::run(p, d_data, total, d_offsets, nfiles, d_cuts, cap,
                            d_cut_offsets, d_count, d_ws, ws_bytes, piece, sms_w, host_data,
                            stream, g_prof_begin, g_prof_end);
  }
  const uint32_t L = pick_segment(p, tuning);
  const uint32_t threads = pick_threads(tuning);
  const Layout l = make_layout(p, total, nfiles, L);
  if (l.imax >= 0xffffffffull) return SEQCDC_ERANGE;
  if (ws_bytes < l.total) return SEQCDC_ECAPACITY;
  if (cap < total / p->min_size + nfiles) return SEQCDC_ECAPACITY;
  if (kind < 0) return SEQCDC_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const WsPtrs w = ws_ptrs(d_ws, l);
  Geom g{d_data, total, d_offsets, nfiles, L, cand_cap(L), g_wait_ns, host_data ? 1u : 0u};
  DevParams dp{p->mode, p->seq_length, p->skip_trigger, p->skip_size,
               (uint32_t)p->min_size, (uint32_t)p->max_size};
  const size_t smem = map_smem_bytes(max_words(L, p->max_size), L);
  if (smem > kSmemBudget) return SEQCDC_ERANGE;
  void (*map_fn)(Geom, DevParams, WsPtrs) =
      threads == 128u ? map_kernel<128, 12>
                      : threads == 512u ? map_kernel<512, 3> : map_kernel<256, 6>;
  if (smem > 48 * 1024 && !smem_configured(threads, smem, map_fn)) return SEQCDC_ECUDA;
  const int sms = sm_count();
  if (sms <= 0) return SEQCDC_ECUDA;
  plan_tiles_kernel<<<(unsigned)l.nftiles, 256, 0, st>>>(g, w);
  plan_scan_kernel<<<(unsigned)l.nftiles, 256, 0, st>>>(g, w, l.nftiles, l.imax);
  if (g_prof_begin) record_event(g_prof_begin, st);
  map_fn<<<(unsigned)l.imax, threads, smem, st>>>(g, dp, w);
  if (g_prof_end) record_event(g_prof_end, st);
  // Warps per resolve block: up to kResolveWarps while their staging areas
  // stay within 96 KiB.
  const size_t rper = 2 * sizeof(uint32_t) * cand_cap(L);
  uint32_t rwarps = (uint32_t)((96 * 1024) / rper);
  rwarps = rwarps < 1 ? 1 : (rwarps > (uint32_t)kResolveWarps ? (uint32_t)kResolveWarps : rwarps);
  const size_t rsmem = rper * rwarps;
  if (rsmem > 48 * 1024 && !resolve_smem_configured(rsmem)) return SEQCDC_ECUDA;
  resolve_kernel<<<(unsigned)((l.imax + rwarps - 1) / rwarps), 32 * rwarps, rsmem, st>>>(g, w);
  const uint64_t vblocks = (l.imax + 255) / 256;
  const unsigned vgrid = (unsigned)(vblocks < 4096 ? vblocks : 4096);
  const unsigned rgrid = (unsigned)(l.imax < 2u * (uint64_t)sms ? l.imax : 2u * (uint64_t)sms);
  for (uint32_t round = 0; round < kRepairRounds; ++round) {
    verify_kernel<<<vgrid, 256, 0, st>>>(g, w, round);
    run_repair_kernel<<<rgrid, threads, smem, st>>>(g, dp, w, round);
  }
  verify_kernel<<<vgrid, 256, 0, st>>>(g, w, kRepairRounds);
  // One block per still-inconsistent file, over a grid of at most 4 per SM
  // (files are taken in strides; almost all have nothing to do).
  const uint64_t rblocks = nfiles ? nfiles : 1;
  const uint64_t rcap = 4u * (uint64_t)sms;
  repair_kernel<<<(unsigned)(rblocks < rcap ? rblocks : rcap), threads, smem, st>>>(g, dp, w);
  count_tiles_kernel<<<(unsigned)l.nitiles, kItemTile, 0, st>>>(w);
  emit_kernel<<<(unsigned)(l.nitiles * kEmitSplit), kItemTile, 0, st>>>(g, w, d_cuts, cap,
                                                          d_cut_offsets, d_count);
  return cudaGetLastError() == cudaSuccess ? SEQCDC_OK : SEQCDC_ECUDA;
}

// ---------------------------------------------------------------------------
// Fixed device scratch for seqcdc_chunk_noalloc().  A file-scope device array
// of SEQCDC_NOALLOC_SCRATCH_BYTES: every GPU that loads this library holds it
// until the process exits.  In host code its name is only a host-side handle;
// the device address is looked up once per device and cached.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[SEQCDC_NOALLOC_SCRATCH_BYTES];

__global__ void copy_status_kernel(const WsHeader *hdr, uint32_t *out) {
  *out = hdr->status;
}

// Device address of g_noalloc_scratch on the current device (set-up on first
// use per device, with that device current).  nullptr on failure.
void *noalloc_scratch_address() {
  static std::mutex mu;
  static void *addr[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    addr[dev] = p;
  }
  return addr[dev];
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI.
// ---------------------------------------------------------------------------
extern "C" {

int seqcdc_params(uint32_t expected_kib, uint32_t mode, seqcdc_params_t *out) {
  if (!out || mode > 1) return SEQCDC_EINVAL;
  // Table I (SeqLength, SkipTrigger, SkipSize); Sec. VI min / max sizes.
  uint32_t seq, trig, skip;
  uint64_t mn;
  switch (expected_kib) {
    case 4: seq = 5; trig = 55; skip = 256; mn = 1024; break;
    case 8: seq = 5; trig = 50; skip = 256; mn = 4096; break;
    case 16: seq = 5; trig = 50; skip = 512; mn = 8192; break;
    default: return SEQCDC_EINVAL;
  }
  out->mode = mode;
  out->seq_length = seq;
  out->skip_trigger = trig;
  out->skip_size = skip;
  out->min_size = mn;
  out->max_size = 2ull * expected_kib * 1024ull;
  return SEQCDC_OK;
}

int seqcdc_validate(const seqcdc_params_t *p) {
  return params_ok(p) ? SEQCDC_OK : SEQCDC_EINVAL;
}

int seqcdc_resolve_tuning(const seqcdc_params_t *p, const seqcdc_tuning_t *tuning,
                          seqcdc_tuning_t *out) {
  if (!params_ok(p) || !out) return SEQCDC_EINVAL;
  out->segment_bytes = pick_segment(p, tuning);
  out->block_threads = pick_threads(tuning);
  out->algorithm = tuning ? tuning->algorithm : SEQCDC_ALGO_AUTO;
  out->piece_bytes = seqcdc_walk::pick_piece(p, tuning);
  return SEQCDC_OK;
}

size_t seqcdc_workspace_size(const seqcdc_params_t *p, uint64_t total_bytes,
                             uint64_t nfiles, const seqcdc_tuning_t *tuning) {
  if (!params_ok(p)) return 0;
  // The path seqcdc_chunk_batch() takes for these sizes; for one file,
  // which seqcdc_chunk() may chunk too, whichever path needs more.
  const size_t as_batch = workspace_for(p, total_bytes, nfiles, tuning, true);
  if (nfiles != 1) return as_batch;
  const size_t as_stream = workspace_for(p, total_bytes, nfiles, tuning, false);
  return as_batch > as_stream ? as_batch : as_stream;
}

int seqcdc_algorithm(const seqcdc_params_t *p, uint64_t total_bytes, uint64_t nfiles,
                     int batch, size_t ws_bytes, const seqcdc_tuning_t *tuning) {
  if (!params_ok(p)) return 0;
  return decide_walk(p, total_bytes, nfiles, batch != 0, ws_bytes, tuning)
             ? (int)SEQCDC_ALGO_WALK : (int)SEQCDC_ALGO_MAP;
}

int seqcdc_chunk(const seqcdc_params_t *p, const uint8_t *d_in, uint64_t n,
                 uint64_t *d_cuts, uint64_t cap, uint64_t *d_count,
                 void *d_ws, size_t ws_bytes, const seqcdc_tuning_t *tuning,
                 void *stream) {
  if (!d_count) return SEQCDC_EINVAL;
  return run(p, d_in, n, nullptr, 1, d_cuts, cap, nullptr, d_count, d_ws,
             ws_bytes, tuning, stream, true);
}

int seqcdc_chunk_batch(const seqcdc_params_t *p, const uint8_t *d_data,
                       uint64_t total_bytes, const uint64_t *d_offsets,
                       uint64_t nfiles, uint64_t *d_cuts, uint64_t cap,
                       uint64_t *d_cut_offsets, void *d_ws, size_t ws_bytes,
                       const seqcdc_tuning_t *tuning, void *stream) {
  if (!d_offsets || !d_cut_offsets) return SEQCDC_EINVAL;
  return run(p, d_data, total_bytes, d_offsets, nfiles, d_cuts, cap,
             d_cut_offsets, nullptr, d_ws, ws_bytes, tuning, stream, true);
}

int seqcdc_chunk_noalloc(const seqcdc_params_t *p, const uint8_t *d_in,
                         uint64_t n, uint64_t *d_cuts, uint64_t cap,
                         uint64_t *d_count, uint32_t *d_status,
                         const seqcdc_tuning_t *tuning, void *stream) {
  if (!d_count || !params_ok(p)) return SEQCDC_EINVAL;
  // The path the call takes with this scratch (AUTO takes the chain walk
  // where the segment map's workspace would not fit), and its workspace.
  const size_t scratch = (size_t)SEQCDC_NOALLOC_SCRATCH_BYTES;
  const size_t need =
      decide_walk(p, n, 1, false, scratch, tuning)
          ? seqcdc_walk::workspace_bytes(p, n, 1, seqcdc_walk::pick_piece(p, tuning))
          : make_layout(p, n, 1, pick_segment(p, tuning)).total;
  if (need > scratch) return SEQCDC_ERANGE;
  void *ws = noalloc_scratch_address();
  if (!ws) return SEQCDC_ECUDA;
  const int rc = run(p, d_in, n, nullptr, 1, d_cuts, cap, nullptr, d_count, ws,
                     (size_t)SEQCDC_NOALLOC_SCRATCH_BYTES, tuning, stream);
  if (rc != SEQCDC_OK || !d_status) return rc;
  copy_status_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const WsHeader *>(ws), d_status);
  return cudaGetLastError() == cudaSuccess ? SEQCDC_OK : SEQCDC_ECUDA;
}

int seqcdc_copy_ranges(void *dst, const void *src, const uint64_t *dst_off,
                       const uint64_t *src_off, const uint64_t *len, uint64_t n,
                       void *stream) {
  if (n == 0) return SEQCDC_OK;
  if (!dst || !src || !dst_off || !src_off || !len) return SEQCDC_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char *d = static_cast<char *>(dst);
  const char *s = static_cast<const char *>(src);
  for (uint64_t i = 0; i < n; ++i) {
    if (!len[i]) continue;
    if (cudaMemcpyAsync(d + dst_off[i], s + src_off[i], len[i], cudaMemcpyDefault, st) !=
        cudaSuccess)
      return SEQCDC_ECUDA;
  }
  return SEQCDC_OK;
}

int seqcdc_status(const void *d_ws, void *stream) {
  if (!d_ws) return SEQCDC_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  if (cudaMemcpyAsync(&v, d_ws, sizeof(v), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SEQCDC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SEQCDC_ECUDA;
  return (int)v;
}

int seqcdc_stats(const void *d_ws, void *stream, uint32_t *out, uint32_t n) {
  if (!d_ws || !out) return SEQCDC_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  WsHeader h;
  if (cudaMemcpyAsync(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return SEQCDC_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SEQCDC_ECUDA;
  for (uint32_t k = 0; k < n && k < 8; ++k) out[k] = h.stats[k];
  return SEQCDC_OK;
}

uint64_t seqcdc_set_wait_limit_ns(uint64_t ns) {
  const uint64_t prev = g_wait_ns;
  g_wait_ns = ns;
  return prev;
}

int seqcdc_profile_events(void *ev_begin, void *ev_end) {
  g_prof_begin = static_cast<cudaEvent_t>(ev_begin);
  g_prof_end = static_cast<cudaEvent_t>(ev_end);
  return SEQCDC_OK;
}

const char *seqcdc_strerror(int status) {
  switch (status) {
    case SEQCDC_OK: return "ok";
    case SEQCDC_EINVAL: return "invalid argument (parameters, pointer or alignment)";
    case SEQCDC_ECAPACITY: return "output capacity or workspace too small";
    case SEQCDC_ECUDA: return "CUDA runtime error";
    case SEQCDC_ETIMEOUT: return "a bounded device-side wait expired";
    case SEQCDC_ERANGE: return "input too large for this library";
    default: return "unknown status";
  }
}

}  // extern "C"
