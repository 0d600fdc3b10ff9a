// walk.cu -- SeqCDC by walking the chunk chain, reading only what it scans.
//
// The sequential chunker of Sec. III looks at few of the input bytes: the
// first min_size - SeqLength bytes of every chunk are never scanned
// (Sec. III.B) and SkipSize bytes are passed over after each skip
// (Sec. III.C).  This path follows the chain the way the paper's scan does,
// one chunk after the other, with a whole warp per scan step: the warp loads
// a 1 KiB window of the scan region (32 bytes per lane), classifies its byte
// pairs into the T, O and E bits of Sec. III.D, and finds the first run end
// and the SkipTrigger-th opposing pair with a ballot and a warp prefix sum.
// Only the windows the chain scans are read from memory.
//
// The chain is sequential, so parallelism comes from many chains at once:
//   plan      split every file into pieces of P bytes (P >= 4 max_size).
//   walk      one warp per piece (longest first) walks the chain from the
//             piece start as if a chunk began there, up to the first cut at
//             or after the piece end (the piece's exit); for a file's first
//             piece this is the true chain.  The warp then walks on from that
//             exit into the file's next piece (the next piece's junction
//             walk) until it reaches a cut of that piece's own walk: the
//             chunk after a cut depends only on the cut, so from the meeting
//             cut on the two chains are the same.
//   verify    a piece's junction started from the exit its predecessor's
//             walk computed; where the predecessor's final exit differs (its
//             own junction never met its walk) the piece is inconsistent.  A
//             file without inconsistent pieces is exact by induction from its
//             start.
//   repair    one warp per file with an inconsistent piece redoes the
//             junctions in order from the first such piece.
//   compact   count each piece's cuts, exclusive scan, copy to the caller's
//             CSR output.
// Input in pinned host memory is read in place over the host link; there the
// bytes that cross bound the walk, and its chunk step (chunk_end_host) loads
// 128 bytes at a time from each scan region's start instead of 1 KiB windows.
//
// Chains started at different positions meet after a few dozen chunks on
// ordinary data, well within a piece.  In long stretches with no run ends
// (constant bytes, where every cut is forced at max_size) they never meet,
// and the repair pass walks those stretches one file at a time.

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "seqcdc.h"
#include "walk.h"

namespace {

constexpr int kWalkThreads = 128;      // walk kernels: four warps per block
// Blocks of the walk kernels resident per SM that the register budget is
// sized for: 16 blocks of 4 warps, 32 registers per thread without spills
// (the walks are bound by latency and issue; 64 chains in flight per SM).
#ifndef SEQCDC_WALK_MIN_BLOCKS
#define SEQCDC_WALK_MIN_BLOCKS 16
#endif
constexpr int kWalkMinBlocks = SEQCDC_WALK_MIN_BLOCKS;
// Lanes (16 bytes each) the walk over host-resident input loads at a time.
#ifndef SEQCDC_HOST_GROW
#define SEQCDC_HOST_GROW 8
#endif
constexpr int kFileTile = 1024;        // files per plan block
constexpr int kPieceTile = 32;         // pieces per compaction tile (8 warps copy 4 each)
constexpr int kEmitThreads = 256;
constexpr uint32_t kUnmerged = 0xFFFFFFFFu;
constexpr uint32_t kNoBad = 0xFFFFFFFFu;
constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kDefaultPiece = 768u << 10;
// Rounds of verify + parallel run repair before the sequential repair.
constexpr uint32_t kWalkRepairRounds = 3;

// Workspace header: status and statistics at the offsets seqcdc_status and
// seqcdc_stats read.
struct WalkHeader {
  uint32_t status;         // 0 or a SEQCDC_* error code
  uint32_t ticket;         // piece-walk queue head
  uint32_t npieces;
  uint32_t stats[8];
  uint32_t nlong, nshort;  // walk-order fill counters
  uint32_t nruns[kWalkRepairRounds];  // runs of inconsistent pieces found by each verify round
  uint32_t runq[kWalkRepairRounds];   // run queue head of each parallel repair round
  uint32_t pad[51 - 2 * kWalkRepairRounds];
};
static_assert(sizeof(WalkHeader) == 256, "walk header is 256 bytes");

enum : uint32_t {
  WS_PIECES = 0,        // pieces walked
  WS_SPEC_CHUNKS = 1,   // chunks found by the spec walks
  WS_JUNCTIONS = 2,     // junction walks
  WS_JCHUNKS = 3,       // chunks the junction walks took before meeting
  WS_UNMERGED = 4,      // junction walks that left their piece without meeting
  WS_INCONSISTENT = 5,  // pieces whose junction input was wrong
  WS_REPAIRED = 6,      // junction walks redone by the repair pass
  WS_WINDOWS = 7,       // 1 KiB windows the walks loaded (32-byte sectors when
                        // the input is read in place from host memory)
};

struct WGeom {
  const uint8_t *data;
  uint64_t total;
  const uint64_t *offsets;  // nullptr: one stream of `total` bytes
  uint64_t nfiles;
  uint32_t P;               // piece bytes
  uint32_t fullcap;         // list entries of a full piece (P / min_size + 3)
  uint32_t host;            // the data is pinned host memory read in place
};

struct WPtrs {
  WalkHeader *hdr;
  uint32_t *piece_base;  // nfiles + 1: first piece of each file
  uint64_t *list_base;   // nfiles + 1: first list entry of each file
  uint32_t *ftile;       // per plan tile: pieces of its files
  uint64_t *ftile_l;     // per plan tile: list entries of its files
  uint32_t *piece_file;  // per piece
  uint32_t *order;       // per piece: walk order (long pieces first)
  uint32_t *spec_n;      // per piece: cuts of its spec walk (the exit last)
  uint32_t *sdone;       // per piece: 1 once its spec walk's cuts are published
  uint32_t *spec;        // list entries: spec-walk cuts, relative to the piece start
  uint32_t *jin;         // per piece: where its junction walk started (relative)
  uint32_t *jn;          // per piece: junction cuts before the meeting cut
  uint32_t *jm;          // per piece: index of the meeting cut in spec, or kUnmerged
  uint32_t *jexit;       // per piece: exit of a junction walk that did not meet
  uint32_t *jcut;        // list entries: junction cuts, relative to the piece start
  uint32_t *first_bad;   // per file: first inconsistent piece
  uint32_t *count;       // per piece: cuts it owns (c with start < c <= end)
  uint32_t *ctile;       // per compaction tile: their sum
  uint32_t *bad;         // per piece: round + 1 if the verify of that round found it inconsistent
  uint32_t *runs;        // first pieces of the runs of inconsistent pieces (one round's list)
  uint32_t *claim;       // per piece: the last repair round (round + 1) that owns it
};

__device__ __forceinline__ uint64_t wfile_start(const WGeom &g, uint64_t f) {
  return g.offsets ? g.offsets[f] : 0;
}
__device__ __forceinline__ uint64_t wfile_end(const WGeom &g, uint64_t f) {
  return g.offsets ? g.offsets[f + 1] : g.total;
}

// List entries a piece of `len` bytes reserves: its cuts in (start, end] are
// at least min_size apart except the file's last, plus the exit.
__host__ __device__ __forceinline__ uint32_t list_cap(uint32_t len, uint32_t mn) {
  return len / mn + 3;
}

__device__ __forceinline__ uint64_t file_lists(uint64_t n, uint32_t P, uint32_t fullcap,
                                               uint32_t mn) {
  const uint64_t tail = n % P;
  return (n / P) * fullcap + (tail ? list_cap((uint32_t)tail, mn) : 0u);
}

struct Piece {
  uint64_t ps;    // absolute start
  uint64_t fend;  // absolute end of its file
  uint64_t lb;    // first list entry
  uint32_t len;   // bytes
  uint32_t kl;    // index within its file
  uint32_t cap;   // list entries
  uint32_t file;
};

__device__ __forceinline__ Piece piece_of(const WGeom &g, const WPtrs &w, const DevParams &p,
                                          uint32_t k) {
  Piece pc;
  pc.file = w.piece_file[k];
  pc.kl = k - w.piece_base[pc.file];
  const uint64_t fs = wfile_start(g, pc.file);
  pc.fend = wfile_end(g, pc.file);
  pc.ps = fs + (uint64_t)pc.kl * g.P;
  const uint64_t rest = pc.fend - pc.ps;
  pc.len = (uint32_t)(rest < g.P ? rest : g.P);
  pc.lb = w.list_base[pc.file] + (uint64_t)pc.kl * g.fullcap;
  pc.cap = list_cap(pc.len, p.mn);
  return pc;
}

__device__ __forceinline__ void set_status(WalkHeader *h, uint32_t code) {
  atomicCAS(&h->status, 0u, code);
}

// ---------------------------------------------------------------------------
// Plan: pieces and list entries per file, their prefix sums, walk order.
// ---------------------------------------------------------------------------
__global__ void wplan_tiles_kernel(WGeom g, DevParams p, WPtrs w) {
  __shared__ uint32_t red[32];
  __shared__ uint64_t red_l[32];
  const uint64_t f0 = (uint64_t)blockIdx.x * kFileTile;
  uint32_t sum = 0;
  uint64_t sum_l = 0;
  for (uint64_t f = f0 + threadIdx.x; f < f0 + kFileTile && f < g.nfiles; f += blockDim.x) {
    const uint64_t n = wfile_end(g, f) - wfile_start(g, f);
    sum += (uint32_t)((n + g.P - 1) / g.P);
    sum_l += file_lists(n, g.P, g.fullcap, p.mn);
  }
  for (int d = 16; d; d >>= 1) {
    sum += __shfl_down_sync(kFull, sum, d);
    sum_l += __shfl_down_sync(kFull, sum_l, d);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5] = sum;
    red_l[threadIdx.x >> 5] = sum_l;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    uint64_t s_l = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      s += red[k];
      s_l += red_l[k];
    }
    w.ftile[blockIdx.x] = s;
    w.ftile_l[blockIdx.x] = s_l;
  }
}

// Exclusive block scan of one 64-bit value per thread.
__device__ uint64_t block_excl_scan64(uint64_t v, uint64_t *scratch, uint64_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  uint64_t x = v;
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t y = __shfl_up_sync(kFull, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint64_t s = lane < nwarps ? scratch[lane] : 0ull;
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(kFull, s, d);
      if (lane >= d) s += y;
    }
    if (lane < nwarps) scratch[lane] = s;
  }
  __syncthreads();
  const uint64_t warp_off = warp ? scratch[warp - 1] : 0ull;
  *total = scratch[nwarps - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void wplan_scan_kernel(WGeom g, DevParams p, WPtrs w, uint64_t nftiles) {
  __shared__ uint32_t scratch[32];
  __shared__ uint64_t scratch_l[32];
  __shared__ uint32_t s_prefix;
  __shared__ uint64_t s_prefix_l;
  uint32_t part = 0;
  uint64_t part_l = 0;
  for (uint64_t t = threadIdx.x; t < blockIdx.x; t += blockDim.x) {
    part += w.ftile[t];
    part_l += w.ftile_l[t];
  }
  for (int d = 16; d; d >>= 1) {
    part += __shfl_down_sync(kFull, part, d);
    part_l += __shfl_down_sync(kFull, part_l, d);
  }
  if ((threadIdx.x & 31) == 0) {
    scratch[threadIdx.x >> 5] = part;
    scratch_l[threadIdx.x >> 5] = part_l;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    uint64_t s_l = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      s += scratch[k];
      s_l += scratch_l[k];
    }
    s_prefix = s;
    s_prefix_l = s_l;
  }
  __syncthreads();
  uint32_t running = s_prefix;
  uint64_t running_l = s_prefix_l;
  const uint64_t f0 = (uint64_t)blockIdx.x * kFileTile;
  for (uint64_t c0 = f0; c0 < f0 + kFileTile; c0 += blockDim.x) {
    const uint64_t f = c0 + threadIdx.x;
    const bool live = f < g.nfiles && f < f0 + kFileTile;
    const uint64_t n = live ? wfile_end(g, f) - wfile_start(g, f) : 0;
    const uint32_t v = live ? (uint32_t)((n + g.P - 1) / g.P) : 0u;
    const uint64_t v_l = live ? file_lists(n, g.P, g.fullcap, p.mn) : 0ull;
    uint32_t tot;
    uint64_t tot_l;
    const uint32_t ex = block_excl_scan(v, scratch, &tot);
    const uint64_t ex_l = block_excl_scan64(v_l, scratch_l, &tot_l);
    if (live) {
      w.piece_base[f] = running + ex;
      w.list_base[f] = running_l + ex_l;
    }
    running += tot;
    running_l += tot_l;
  }
  if (blockIdx.x == nftiles - 1 && threadIdx.x == 0) {
    w.piece_base[g.nfiles] = running;
    w.list_base[g.nfiles] = running_l;
    WalkHeader *h = w.hdr;
    h->status = 0;
    h->ticket = 0;
    h->npieces = running;
    h->nlong = 0;
    h->nshort = 0;
    for (uint32_t q = 0; q < kWalkRepairRounds; ++q) {
      h->nruns[q] = 0;
      h->runq[q] = 0;
    }
    for (int k = 0; k < 8; ++k) h->stats[k] = 0;
  }
  for (uint64_t f = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; f < g.nfiles;
       f += (uint64_t)gridDim.x * blockDim.x)
    w.first_bad[f] = kNoBad;
}

// piece_file of every piece, and the walk order: first (filled from the
// front) every piece of a file with several pieces and every piece of at
// least P/2 bytes, then the short single-piece files (filled from the back).
// The longest walks thus start in the first wave, and a piece's successor
// is walked alongside it, so that its cuts are there when this piece's warp
// walks on into it.
__global__ void wfill_kernel(WGeom g, WPtrs w) {
  const uint32_t np = w.hdr->npieces;
  const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = k < np;
  bool longp = false;
  if (live) {
    // The last file whose first piece is at or before k holds it (an empty
    // file shares its first-piece index with the next file).
    uint64_t a = 0, b = g.nfiles - 1;
    while (a < b) {
      const uint64_t mid = (a + b + 1) >> 1;
      if (w.piece_base[mid] <= k) a = mid; else b = mid - 1;
    }
    w.piece_file[k] = (uint32_t)a;
    w.sdone[k] = 0u;
    w.claim[k] = 0u;
    const uint64_t ps = wfile_start(g, a) + (k - w.piece_base[a]) * (uint64_t)g.P;
    longp = w.piece_base[a + 1] - w.piece_base[a] > 1u ||
            wfile_end(g, a) - ps >= (uint64_t)(g.P >> 1);
  }
  const int lane = threadIdx.x & 31;
  const uint32_t bl = __ballot_sync(kFull, live && longp);
  const uint32_t bs = __ballot_sync(kFull, live && !longp);
  uint32_t base_l = 0, base_s = 0;
  if (lane == 0) {
    if (bl) base_l = atomicAdd(&w.hdr->nlong, (uint32_t)__popc(bl));
    if (bs) base_s = atomicAdd(&w.hdr->nshort, (uint32_t)__popc(bs));
  }
  base_l = __shfl_sync(kFull, base_l, 0);
  base_s = __shfl_sync(kFull, base_s, 0);
  const uint32_t below = (1u << lane) - 1u;
  if (live) {
    if (longp) w.order[base_l + __popc(bl & below)] = (uint32_t)k;
    else w.order[np - 1u - (base_s + __popc(bs & below))] = (uint32_t)k;
  }
}

// ---------------------------------------------------------------------------
// One chunk, one warp.
// ---------------------------------------------------------------------------
// Bits 0 .. n-1 set (n >= 0; 32 and more: all).
__device__ __forceinline__ uint32_t low_bits(int32_t n) {
  return __funnelshift_lc(0xffffffffu, 0u, (uint32_t)(n < 0 ? 0 : n));
}

// A 1 KiB window of input held in registers: 16 bytes per lane in each of
// its two 512-byte halves, starting at the 16-aligned absolute byte `base`.
struct Win {
  uint4 a, b;
};

__device__ __forceinline__ Win load_win(const WGeom &g, uint64_t base) {
  const int lane = threadIdx.x & 31;
  const uint64_t off = base + 16u * lane;
  Win w;
  if (off + 528u <= g.total) {
    w.a = __ldg(reinterpret_cast<const uint4 *>(g.data + off));
    w.b = __ldg(reinterpret_cast<const uint4 *>(g.data + off + 512u));
  } else {
    w.a = load16(g.data, (int64_t)off, g.total);
    w.b = load16(g.data, (int64_t)(off + 512u), g.total);
  }
  return w;
}

template <uint32_t MODE, bool R5>
__device__ uint64_t chunk_end_host(const WGeom &g, const DevParams &p, uint64_t c,
                                   uint64_t fend, uint32_t &secs, bool &ok);

// End of the chunk that starts at absolute byte c of a file ending at fend
// (Sec. III.A-C, Sec. IV): the chunk limit is c + max_size (or the file end);
// the scan starts min_size - SeqLength bytes in; a region ends at its first
// run end (cut right after it) or at its SkipTrigger-th opposing pair, after
// which SkipSize bytes are passed over and a new region starts.  All lanes
// of the warp call this together and get the same result.
//
// A window is 1 KiB loaded at once; a 512-byte half is classified only when
// the scan reaches it.  Lane l's word of a half holds the half's positions
// 16 l .. 16 l + 15 in bits 0..15.  Positions are 32-bit offsets from the
// first window's start.  Only the windows the scan reaches are read: with
// many chains in flight per SM the loads' latency is hidden.  An L2 prefetch
// of the next chunk's likely window on every chunk measured no faster and
// moved three to four times the bytes, so it is taken (`pf`) only where the
// walk waits on memory.  With LAZY (input in host memory) the chunk goes to
// chunk_end_host instead.
template <uint32_t MODE, bool R5, bool LAZY>
__device__ uint64_t chunk_end_warp(const WGeom &g, const DevParams &p, uint64_t c,
                                   uint64_t fend, uint32_t &wins, bool &ok, bool pf = false) {
  if (LAZY) return chunk_end_host<MODE, R5>(g, p, c, fend, wins, ok);
  const int lane = threadIdx.x & 31;
  if (pf) {
    // Ask L2 for 3 KiB where the next chunk's scan most likely starts (its
    // cut is at least min_size on, its scan min_size - SeqLength after that),
    // so that its first window does not wait for HBM.  Used only where the
    // walk is bound by latency rather than issue: once no piece is left to
    // take, and in the repairs (few warps) of input in device memory.
    const uint64_t a = ((c + 2ull * p.mn - p.R) & ~127ull) + 128u * (uint32_t)lane;
    if (lane < 24 && a + 128u <= g.total)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(g.data + a));
  }
  const uint64_t rest = fend - c;
  const uint64_t lim_abs = c + (rest > p.mx ? p.mx : rest);
  const uint64_t r_abs = c + (p.mn > p.R ? p.mn - p.R : 0u);
  if (r_abs + 1 >= lim_abs) return lim_abs;
  const uint64_t cb = r_abs & ~15ull;
  Win cur = load_win(g, cb);
  ++wins;
  const uint32_t lim = (uint32_t)(lim_abs - cb);
  uint32_t r = (uint32_t)(r_abs - cb);
  // A skip past the limit ends the chunk at the limit, so SkipSize can be
  // clamped to it and every position stays below 2^32.
  const uint32_t skip = p.S < lim ? p.S : lim;
  const int32_t lb = 16 * lane;     // the lane's first position in a half
  uint32_t opp = 0;                 // opposing pairs counted in the current region
  uint32_t w0 = 0;                  // window start
  uint32_t carry_b = 0, carry_t = 0;  // byte and T bits before the half (continued region)
  // Every window either ends the chunk, starts a region at least
  // SkipSize + 2 bytes further on, or moves 1 KiB ahead, so a chunk of at
  // most max_size bytes needs fewer windows than this bound.
  const uint32_t max_windows = p.mx + 8u;
  for (uint32_t it = 0; it < max_windows; ++it) {
    if (it) {
      cur = load_win(g, cb + w0);
      ++wins;
    }
    bool fresh = false;  // the next window starts a new region at r
    // A region that starts inside the second half skips classifying the
    // first (its first pair, (r, r + 1), then lies wholly in the second).
    for (int h = (r >= w0 + 512u) ? 1 : 0; h < 2; ++h) {
      const uint32_t hb = w0 + 512u * h;  // half start (< lim)
      const uint4 v = h ? cur.b : cur.a;
      uint32_t prev = __shfl_up_sync(kFull, v.w >> 24, 1);
      if (lane == 0) prev = carry_b;
      uint32_t Tw, Ow;
      classify16(v, prev, MODE, Tw, Ow);
      uint32_t pt = __shfl_up_sync(kFull, Tw, 1);
      if (lane == 0) pt = carry_t;
      // The run ends of this lane's 16 positions look back into the 16 before.
      const uint32_t Ew = run_ends(0u, (Tw << 16) | (pt & 0xffffu), R5 ? 5u : p.R) >> 16;
      carry_b = __shfl_sync(kFull, v.w >> 24, 31);
      carry_t = __shfl_sync(kFull, Tw, 31);
      const uint32_t span = lim - hb;
      const uint32_t hmask = low_bits((int32_t)(span < 1024u ? span : 1024u) - lb);  // pairs j < lim
      bool moved = false;  // a skip moved r past this half
      for (;;) {
        // Region from r: run ends at j >= r + SeqLength - 1 (the whole run
        // after r), opposing pairs (j-1, j) with j >= r + 1, all below lim.
        const int32_t rr = (int32_t)(r - hb);
        const uint32_t em = Ew & hmask & ~low_bits(rr + (int32_t)p.R - 1 - lb);
        const uint32_t om = Ow & hmask & ~low_bits(rr + 1 - lb);
        const uint32_t eb = __ballot_sync(kFull, em != 0u);
        uint32_t need = 0;  // nonzero: the need-th opposing pair here fires a skip
        if (eb) {
          const int el = __ffs(eb) - 1;
          const uint32_t ebit = __ffs(__shfl_sync(kFull, em, el)) - 1;
          if (p.T) {
            const uint32_t ob = lane < el ? om : (lane == el ? (om & ((1u << ebit) - 1u)) : 0u);
            const uint32_t before = __reduce_add_sync(kFull, (uint32_t)__popc(ob));
            if (opp + before >= p.T) need = p.T - opp;
          }
          if (!need) return cb + hb + 16u * el + ebit + 1u;
        } else if (p.T) {
          const uint32_t tot = __reduce_add_sync(kFull, (uint32_t)__popc(om));
          if (opp + tot >= p.T) need = p.T - opp;
          else opp += tot;
        }
        if (!need) break;  // the region goes on past this half
        // Skip: the need-th opposing pair fires; bytes after it up to
        // SkipSize are passed over and the next region starts after them.
        const uint32_t cnt = __popc(om);
        uint32_t sc = cnt;
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t y = __shfl_up_sync(kFull, sc, d);
          if (lane >= d) sc += y;
        }
        const int ol = __ffs(__ballot_sync(kFull, sc >= need)) - 1;
        // The k-th set bit of lane ol's word: lane t checks bit t.
        const uint32_t word = __shfl_sync(kFull, om, ol);
        const uint32_t kth = __shfl_sync(kFull, need - (sc - cnt), ol);
        const bool hit = ((word >> lane) & 1u) &&
                         (uint32_t)__popc(word & (0xffffffffu >> (31 - lane))) == kth;
        const uint32_t bp = __ffs(__ballot_sync(kFull, hit)) - 1;
        r = hb + 16u * ol + bp + 1u + skip;
        opp = 0;
        if (r + 1 >= lim) return cb + lim;
        if (r + 1 < hb + 512u) continue;  // the next region starts in this half
        moved = true;
        break;
      }
      if (!moved) {
        // No event: the region continues into the bytes after this half.
        if (hb + 512u >= lim) return cb + lim;
        continue;  // next half, or (after half 1) the next window
      }
      if (h == 0 && r + 1 < w0 + 1024u) continue;  // the new region starts in half 1
      fresh = true;
      break;
    }
    if (fresh) {
      w0 = r & ~15u;
      carry_b = 0;
      carry_t = 0;
    } else {
      w0 += 1024u;
    }
  }
  ok = false;
  return cb + lim;
}

// End of the chunk that starts at absolute byte c, as chunk_end_warp, for
// input read in place from host memory, where the bytes that cross the host
// link bound the walk and instructions are cheap.  A scan step covers 512
// bytes from the region's start (16 per lane), but loads them 128 bytes
// (eight lanes) at a time and decides the region on what it has loaded: it
// loads more only while no run end or skip has shown up, and never the bytes
// before the region's start.  `secs` counts the 32-byte sectors read.
template <uint32_t MODE, bool R5>
__device__ uint64_t chunk_end_host(const WGeom &g, const DevParams &p, uint64_t c,
                                   uint64_t fend, uint32_t &secs, bool &ok) {
  constexpr uint32_t kGrow = SEQCDC_HOST_GROW;  // lanes loaded per step
  const int lane = threadIdx.x & 31;
  const uint64_t rest = fend - c;
  const uint64_t lim_abs = c + (rest > p.mx ? p.mx : rest);
  const uint64_t r_abs = c + (p.mn > p.R ? p.mn - p.R : 0u);
  if (r_abs + 1 >= lim_abs) return lim_abs;
  const uint64_t cb = r_abs & ~15ull;  // positions below are relative to cb
  const uint32_t lim = (uint32_t)(lim_abs - cb);
  uint32_t r = (uint32_t)(r_abs - cb);
  const uint32_t skip = p.S < lim ? p.S : lim;
  const int32_t lb = 16 * lane;
  uint32_t opp = 0;                   // opposing pairs of the region before this step
  uint32_t hb = r & ~15u;             // step start
  uint32_t carry_b = 0, carry_t = 0;  // byte and T bits before the step (continued region)
  // Each step ends the chunk, moves the region start SkipSize + 2 or more
  // bytes on, or moves 512 bytes on; each pass of the inner loop loads eight
  // more lanes or handles a skip.
  for (uint32_t it = 0; it < p.mx + 8u; ++it) {
    const uint32_t span = lim - hb;   // positions of the step below lim: [0, span)
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    uint32_t Tw = 0, Ow = 0;
    uint32_t have = 0;                // lanes loaded
    uint32_t upto = 0;                // lanes decided on: [0, upto)
    bool next = false;                // the region goes on into the next step
    for (uint32_t pass = 0; pass < 64u + p.mx; ++pass) {
      const int32_t rr = (int32_t)(r - hb);  // region start in the step (< 0: continued)
      const uint32_t fl = rr > 0 ? (uint32_t)rr >> 4 : 0u;
      if (upto <= fl) upto = min(32u, fl + kGrow);
      const bool need = (uint32_t)lane >= fl && (uint32_t)lane < upto &&
                        !((have >> lane) & 1u) && lb < (int32_t)span;
      if (need) {
        const uint64_t off = cb + hb + (uint32_t)lb;
        v = off + 16u <= g.total ? __ldg(reinterpret_cast<const uint4 *>(g.data + off))
                                 : load16(g.data, (int64_t)off, g.total);
      }
      const uint32_t nb = __ballot_sync(kFull, need);
      if (nb) {
        have |= nb;
        secs += __popc((nb | (nb >> 1)) & 0x55555555u);
        uint32_t prev = __shfl_up_sync(kFull, v.w >> 24, 1);
        if (lane == 0) prev = carry_b;
        classify16(v, prev, MODE, Tw, Ow);
      }
      uint32_t pt = __shfl_up_sync(kFull, Tw, 1);
      if (lane == 0) pt = carry_t;
      const uint32_t Ew = run_ends(0u, (Tw << 16) | (pt & 0xffffu), R5 ? 5u : p.R) >> 16;
      // Positions decided on: the lanes up to `upto`, below lim, from the region on.
      const uint32_t vmask = (uint32_t)lane < upto ? low_bits((int32_t)span - lb) & 0xffffu : 0u;
      const uint32_t em = Ew & vmask & ~low_bits(rr + (int32_t)p.R - 1 - lb);
      const uint32_t om = Ow & vmask & ~low_bits(rr + 1 - lb);
      const bool whole = upto == 32u || 16u * upto >= span;  // the step seen to its end
      const uint32_t eb = __ballot_sync(kFull, em != 0u);
      uint32_t need_k = 0;  // nonzero: the need_k-th opposing pair here fires a skip
      if (eb) {
        const int el = __ffs(eb) - 1;
        const uint32_t ebit = __ffs(__shfl_sync(kFull, em, el)) - 1;
        if (p.T) {
          const uint32_t ob = lane < el ? om : (lane == el ? (om & ((1u << ebit) - 1u)) : 0u);
          const uint32_t before = __reduce_add_sync(kFull, (uint32_t)__popc(ob));
          if (opp + before >= p.T) need_k = p.T - opp;
        }
        if (!need_k) return cb + hb + 16u * el + ebit + 1u;
      } else if (p.T) {
        const uint32_t tot = __reduce_add_sync(kFull, (uint32_t)__popc(om));
        if (opp + tot >= p.T) {
          need_k = p.T - opp;
        } else if (whole) {
          opp += tot;  // the region goes on past this step
          next = true;
          break;
        }
      } else if (whole) {
        next = true;
        break;
      }
      if (!need_k) {  // nothing decided yet: eight more lanes
        upto = min(32u, upto + kGrow);
        continue;
      }
      // Skip: the need_k-th opposing pair fires; the next region starts
      // SkipSize bytes after it.
      const uint32_t cnt = __popc(om);
      uint32_t sc = cnt;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, sc, d);
        if (lane >= d) sc += y;
      }
      const int ol = __ffs(__ballot_sync(kFull, sc >= need_k)) - 1;
      const uint32_t word = __shfl_sync(kFull, om, ol);
      const uint32_t kth = __shfl_sync(kFull, need_k - (sc - cnt), ol);
      const bool hit = ((word >> lane) & 1u) &&
                       (uint32_t)__popc(word & (0xffffffffu >> (31 - lane))) == kth;
      const uint32_t bp = __ffs(__ballot_sync(kFull, hit)) - 1;
      r = hb + 16u * ol + bp + 1u + skip;
      opp = 0;
      if (r + 1 >= lim) return cb + lim;
      if (r + 1 >= hb + 512u) break;  // the next region starts in a later step
      // else the next region starts in this step: decided on what is loaded,
      // its lanes loaded as it needs them
    }
    if (next) {
      if (hb + 512u >= lim) return cb + lim;  // no run end before the limit
      carry_b = __shfl_sync(kFull, v.w >> 24, 31);
      carry_t = __shfl_sync(kFull, Tw, 31);
      hb += 512u;
    } else {
      hb = r & ~15u;  // a fresh step at the new region's start
      carry_b = 0;
      carry_t = 0;
    }
  }
  ok = false;
  return cb + lim;
}

// ---------------------------------------------------------------------------
// Junction walks.
// ---------------------------------------------------------------------------
// Exit of piece k as its current results give it: the last cut of its spec
// walk if its junction met that walk, else the junction walk's exit.
__device__ __forceinline__ uint32_t exit_of(const WPtrs &w, uint32_t k, uint64_t lb) {
  return w.jm[k] != kUnmerged ? w.spec[lb + w.spec_n[k] - 1u] : w.jexit[k];
}

// Index of the first of sp[q..ns) that is >= v (the warp reads 32 at a time;
// the list increases).  Reads bypass L1: the list may have been written
// during this kernel by another SM.
__device__ __forceinline__ uint32_t seek(const uint32_t *sp, uint32_t ns, uint32_t q,
                                         uint32_t v) {
  const int lane = threadIdx.x & 31;
  for (uint32_t s = 0; s <= ns / 32u + 1u; ++s) {
    const uint32_t e = q + lane < ns ? __ldcg(sp + q + lane) : kFull;
    const uint32_t below = __ballot_sync(kFull, e < v);
    q += __popc(below);
    if (below != kFull) break;
  }
  return q;
}

// Walk piece k's chain from x (relative to the piece start) until it reaches
// a cut of the piece's spec walk or leaves the piece; record where it
// started, the cuts before the meeting cut, the meeting index or the exit.
// With `done` set, the piece's spec walk may still be running (another warp):
// its cuts are compared once done[k] is set, the cuts walked before that
// first, in order.  Returns whether the walk met the spec walk.
template <uint32_t MODE, bool R5, bool LAZY>
__device__ bool junction_walk(const WGeom &g, const DevParams &p, const WPtrs &w,
                              uint32_t k, const Piece &pc, uint32_t x, const uint32_t *done,
                              uint32_t &chunks, uint32_t &wins, bool &ok, bool pf = false) {
  const int lane = threadIdx.x & 31;
  const uint32_t *sp = w.spec + pc.lb;
  uint32_t *jc = w.jcut + pc.lb;
  bool have = done == nullptr;
  uint32_t ns = have ? __ldcg(w.spec_n + k) : 0u;
  uint32_t q = 0, n = 0, checked = 0, jm = kUnmerged, jexit = 0;
  uint32_t rel = x;
  if (x == 0) {
    jm = 0;  // the spec walk starts at the input itself
  } else {
    bool fin = false;
    for (uint32_t it = 0; it <= pc.cap && !fin; ++it) {
      if (!have) {
        uint32_t f = 0;
        if (lane == 0) f = ld_acquire(done + k);
        have = __shfl_sync(kFull, f, 0) != 0u;
        if (have) {
          ns = __ldcg(w.spec_n + k);
          __syncwarp();
          for (; checked < n; ++checked) {  // cuts walked before the spec walk was known
            const uint32_t u = __ldcg(jc + checked);
            q = seek(sp, ns, q, u);
            if (q < ns && __ldcg(sp + q) == u) {
              jm = q;
              n = checked;
              fin = true;
              break;
            }
          }
          if (fin) break;
        }
      }
      if (have) {
        q = seek(sp, ns, q, rel);
        if (q < ns && __ldcg(sp + q) == rel) {
          jm = q;
          break;
        }
      }
      if (rel >= pc.len) {
        jexit = rel;
        if (rel == pc.len) {  // a cut exactly at the piece end belongs to it
          if (n < pc.cap) { if (lane == 0) jc[n] = rel; ++n; } else ok = false;
        }
        fin = true;
        break;
      }
      if (n < pc.cap) {
        if (lane == 0) jc[n] = rel;
        ++n;
      } else {
        ok = false;
        fin = true;
        break;
      }
      if (have) checked = n;
      rel = (uint32_t)(chunk_end_warp<MODE, R5, LAZY>(g, p, pc.ps + rel, pc.fend, wins, ok, pf) -
                       pc.ps);
      ++chunks;
    }
    if (!fin && jm == kUnmerged) ok = false;
  }
  if (lane == 0) {
    w.jin[k] = x;
    w.jn[k] = n;
    w.jm[k] = jm;
    w.jexit[k] = jexit;
  }
  __syncwarp();
  return jm != kUnmerged;
}

// ---------------------------------------------------------------------------
// Piece walks: one warp per piece, longest first.  A warp walks its piece's
// chain from the piece start (the spec walk), publishes it, and then walks
// on from the exit into the file's next piece as that piece's junction walk:
// the exit is where the true chain enters the next piece whenever this
// piece's own junction met its spec walk.
// ---------------------------------------------------------------------------
template <uint32_t MODE, bool R5, bool LAZY>
__global__ void __launch_bounds__(kWalkThreads, kWalkMinBlocks)
walk_kernel(WGeom g, DevParams p, WPtrs w) {
  const int lane = threadIdx.x & 31;
  const uint32_t np = w.hdr->npieces;
  uint32_t pieces = 0, chunks = 0, wins = 0, walks = 0, jchunks = 0, unmerged = 0;
  bool ok = true;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&w.hdr->ticket, 1u);
    t = __shfl_sync(kFull, t, 0);
    if (t >= np) break;
    const uint32_t k = w.order[t];
    const Piece pc = piece_of(g, w, p, k);
    const uint64_t pe = pc.ps + pc.len;
    uint32_t *out = w.spec + pc.lb;
    uint64_t c = pc.ps;
    uint32_t n = 0;
    bool pf = false;  // prefetch, once every piece is taken (see below)
    do {
      if (!LAZY && !pf && (n & 7u) == 0u) {
        uint32_t drained = 0;
        if (lane == 0) drained = __ldcg(&w.hdr->ticket) >= np ? 1u : 0u;
        pf = __shfl_sync(kFull, drained, 0) != 0u;
      }
      c = chunk_end_warp<MODE, R5, LAZY>(g, p, c, pc.fend, wins, ok, pf);
      if (n < pc.cap) {
        if (lane == 0) out[n] = (uint32_t)(c - pc.ps);
        ++n;
      } else {
        ok = false;
        break;
      }
    } while (c < pe);
    if (lane == 0) {
      w.spec_n[k] = n;
      if (pc.kl == 0) {  // a file's first piece: its spec walk is its chain
        w.jin[k] = 0;
        w.jn[k] = 0;
        w.jm[k] = 0;
        w.jexit[k] = 0;
      }
      __threadfence();
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(w.sdone + k), "r"(1u) : "memory");
    }
    __syncwarp();
    ++pieces;
    chunks += n;
    if (k + 1 < w.piece_base[pc.file + 1]) {
      const Piece pn = piece_of(g, w, p, k + 1);
      // Once every piece is taken the SMs empty out and the walks left
      // wait on memory rather than on issue: prefetch then.
      if (!LAZY && !pf) {
        uint32_t drained = 0;
        if (lane == 0) drained = __ldcg(&w.hdr->ticket) >= np ? 1u : 0u;
        pf = __shfl_sync(kFull, drained, 0) != 0u;
      }
      const bool met = junction_walk<MODE, R5, LAZY>(g, p, w, k + 1, pn, (uint32_t)(c - pn.ps), w.sdone,
                                     jchunks, wins, ok, pf);
      ++walks;
      unmerged += met ? 0u : 1u;
    }
  }
  if (lane == 0) {
    atomicAdd(&w.hdr->stats[WS_PIECES], pieces);
    atomicAdd(&w.hdr->stats[WS_SPEC_CHUNKS], chunks);
    atomicAdd(&w.hdr->stats[WS_WINDOWS], wins);
    atomicAdd(&w.hdr->stats[WS_JUNCTIONS], walks);
    atomicAdd(&w.hdr->stats[WS_JCHUNKS], jchunks);
    atomicAdd(&w.hdr->stats[WS_UNMERGED], unmerged);
    if (!ok) set_status(w.hdr, SEQCDC_ECAPACITY);
  }
}

// ---------------------------------------------------------------------------
// Verify and repair.
// ---------------------------------------------------------------------------
// Whether piece k (not a file's first) was walked from a wrong entry: its
// junction started somewhere other than its predecessor's exit.
__device__ __forceinline__ bool inconsistent(const WGeom &g, const WPtrs &w, uint32_t k,
                                             uint32_t f, uint32_t kl) {
  const uint64_t lb_prev = w.list_base[f] + (uint64_t)(kl - 1u) * g.fullcap;
  return exit_of(w, k - 1u, lb_prev) - g.P != w.jin[k];
}

// Round `round` < kWalkRepairRounds: flag the inconsistent pieces and list
// the first piece of every maximal run of them for the parallel repair.
// Round kWalkRepairRounds: record each file's first inconsistent piece for
// the sequential repair.
__global__ void wverify_kernel(WGeom g, DevParams p, WPtrs w, uint32_t round) {
  const uint32_t np = w.hdr->npieces;
  uint32_t bad = 0;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < np;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t f = w.piece_file[k];
    const uint32_t kl = (uint32_t)k - w.piece_base[f];
    const bool is_bad = kl > 0 && inconsistent(g, w, (uint32_t)k, f, kl);
    if (round < kWalkRepairRounds) {
      w.bad[k] = is_bad ? round + 1u : 0u;
      if (is_bad && (kl == 1 || !inconsistent(g, w, (uint32_t)k - 1u, f, kl - 1u))) {
        // A run starts here: it and the piece before it (whose exit the run's
        // repair starts from) belong to this round's repair of the run.
        atomicMax(&w.claim[k], round + 1u);
        atomicMax(&w.claim[k - 1], round + 1u);
        w.runs[atomicAdd(&w.hdr->nruns[round], 1u)] = (uint32_t)k;
      }
    } else if (is_bad) {
      atomicMin(&w.first_bad[f], (uint32_t)k);
    }
    bad += is_bad ? 1u : 0u;
  }
  for (int d = 16; d; d >>= 1) bad += __shfl_down_sync(kFull, bad, d);
  if (round == 0 && (threadIdx.x & 31) == 0 && bad)
    atomicAdd(&w.hdr->stats[WS_INCONSISTENT], bad);
}

// Parallel repair: one warp per run of inconsistent pieces (from the list of
// this round), pieces in order: each piece whose junction input differs from
// its predecessor's exit walks again from that exit.  Past the end of its
// run the warp goes on while its new exits keep changing the next piece's
// input (stretches where every piece's own walk agrees with its neighbours'
// but not with the true chain, such as runs of equal bytes or ramps), taking
// each such piece by raising its claim to this round; it stops at a piece
// already claimed this round.  Every run's first piece and the piece before
// it are claimed by the verify, so each piece has at most one writer per
// round, and the piece a run's repair starts from is written by nobody.
// What a round leaves inconsistent the next round's verify lists again.
template <uint32_t MODE, bool R5>
__global__ void __launch_bounds__(kWalkThreads)
wrun_repair_kernel(WGeom g, DevParams p, WPtrs w, uint32_t round) {
  const int lane = threadIdx.x & 31;
  const uint32_t nruns = w.hdr->nruns[round];
  if (nruns == 0) return;  // the usual case once the chains are consistent
  const uint32_t tag = round + 1u;
  uint32_t redone = 0, chunks = 0, wins = 0;
  bool ok = true;
  for (;;) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(&w.hdr->runq[round], 1u);
    t = __shfl_sync(kFull, t, 0);
    if (t >= nruns) break;
    const uint32_t a = w.runs[t];
    const uint32_t kend = w.piece_base[w.piece_file[a] + 1];
    bool in_run = true;
    for (uint32_t k = a; k < kend; ++k) {
      const Piece pc = piece_of(g, w, p, k);
      const uint32_t x = exit_of(w, k - 1u, pc.lb - g.fullcap) - g.P;
      if (in_run && (k == a || w.bad[k] == tag)) {
        if (x == w.jin[k]) continue;
      } else {
        in_run = false;
        if (x == w.jin[k]) break;  // the chain agrees from here on
        uint32_t old = 0;
        if (lane == 0) old = atomicMax(&w.claim[k], tag);
        if (__shfl_sync(kFull, old, 0) >= tag) break;  // another run's piece
      }
      junction_walk<MODE, R5, false>(g, p, w, k, pc, x, nullptr, chunks, wins, ok, !g.host);
      ++redone;
    }
  }
  if (lane == 0) {
    if (redone) atomicAdd(&w.hdr->stats[WS_REPAIRED], redone);
    if (!ok) set_status(w.hdr, SEQCDC_ECAPACITY);
  }
}

// One warp per file (files taken in strides): from the first inconsistent
// piece on, every piece whose junction input differs from its predecessor's
// exit walks again from that exit.  Pieces are taken in order, so each input
// is the true exit of the piece before.
template <uint32_t MODE, bool R5>
__global__ void __launch_bounds__(kWalkThreads)
wrepair_kernel(WGeom g, DevParams p, WPtrs w) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t redone = 0, chunks = 0, wins = 0;
  bool ok = true;
  for (uint64_t f = warp; f < g.nfiles; f += nwarps) {
    const uint32_t kb = w.first_bad[f];
    if (kb == kNoBad) continue;
    const uint32_t kend = w.piece_base[f + 1];
    for (uint32_t k = kb; k < kend; ++k) {
      const Piece pc = piece_of(g, w, p, k);
      const uint32_t x = exit_of(w, k - 1u, pc.lb - g.fullcap) - g.P;
      if (x == w.jin[k]) continue;
      junction_walk<MODE, R5, false>(g, p, w, k, pc, x, nullptr, chunks, wins, ok, !g.host);
      ++redone;
    }
  }
  if (lane == 0) {
    if (redone) atomicAdd(&w.hdr->stats[WS_REPAIRED], redone);
    if (!ok) set_status(w.hdr, SEQCDC_ECAPACITY);
  }
}

// ---------------------------------------------------------------------------
// Compaction.
// ---------------------------------------------------------------------------
// Cuts piece k owns: its junction cuts, then its spec cuts from the meeting
// cut on that lie at or before the piece end.
__device__ __forceinline__ uint32_t owned_cuts(const WPtrs &w, uint32_t k, const Piece &pc) {
  const uint32_t n = w.jn[k], jm = w.jm[k];
  if (jm == kUnmerged) return n;
  const uint32_t ns = w.spec_n[k];
  const uint32_t nle = ns - (w.spec[pc.lb + ns - 1u] > pc.len ? 1u : 0u);
  return n + (nle > jm ? nle - jm : 0u);
}

__global__ void wcount_kernel(WGeom g, DevParams p, WPtrs w) {
  __shared__ uint32_t red[32];
  const uint32_t np = w.hdr->npieces;
  const uint64_t k = (uint64_t)blockIdx.x * kPieceTile + threadIdx.x;
  uint32_t v = 0;
  if (threadIdx.x < kPieceTile && k < np) {
    const Piece pc = piece_of(g, w, p, (uint32_t)k);
    v = owned_cuts(w, (uint32_t)k, pc);
    w.count[k] = v;
  }
  for (int d = 16; d; d >>= 1) v += __shfl_down_sync(kFull, v, d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
    w.ctile[blockIdx.x] = s;
  }
}

__global__ void wemit_kernel(WGeom g, DevParams p, WPtrs w, uint64_t *d_cuts, uint64_t cap,
                             uint64_t *d_cut_offsets, uint64_t *d_count) {
  __shared__ uint32_t scratch[32];
  __shared__ uint64_t red64[32];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t offs[kPieceTile + 1];
  const uint32_t np = w.hdr->npieces;
  const uint64_t lo = (uint64_t)blockIdx.x * kPieceTile;
  uint64_t part = 0;
  for (uint64_t t = threadIdx.x; t < blockIdx.x; t += blockDim.x) part += w.ctile[t];
  for (int d = 16; d; d >>= 1) part += __shfl_down_sync(kFull, part, d);
  if ((threadIdx.x & 31) == 0) red64[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t s = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red64[q];
    s_prefix = s;
  }
  __syncthreads();
  const uint64_t i = lo + threadIdx.x;
  const uint32_t c = (threadIdx.x < kPieceTile && i < np) ? w.count[i] : 0u;
  uint32_t tot;
  const uint32_t ex = block_excl_scan(c, scratch, &tot);
  if (threadIdx.x < kPieceTile) offs[threadIdx.x] = ex;
  if (threadIdx.x == 0) offs[kPieceTile] = tot;
  __syncthreads();
  const uint64_t prefix = s_prefix;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = warp; it < kPieceTile; it += blockDim.x >> 5) {
    const uint64_t k = lo + it;
    if (k >= np) break;
    const uint32_t n = w.count[k];
    const uint64_t at = prefix + offs[it];
    if (at + n > cap) {  // cannot happen for a correct cut list; never write past cap
      if (lane == 0) set_status(w.hdr, SEQCDC_ECAPACITY);
      continue;
    }
    const Piece pc = piece_of(g, w, p, (uint32_t)k);
    const uint64_t fbase = (uint64_t)pc.kl * g.P;  // piece start, file-relative
    const uint32_t nj = w.jn[k], jm = w.jm[k];
    const uint32_t *jc = w.jcut + pc.lb;
    const uint32_t *sp = w.spec + pc.lb + (jm == kUnmerged ? 0u : jm);
    uint64_t *dst = d_cuts + at;
    for (uint32_t j = lane; j < n; j += 32)
      dst[j] = fbase + (j < nj ? jc[j] : sp[j - nj]);
  }
  // CSR offsets of the files whose first piece index falls in [lo, lo+tile).
  const uint64_t hi = lo + kPieceTile;
  if (lo <= np) {
    uint64_t a = 0, b = g.nfiles + 1;  // lower_bound(piece_base, lo)
    while (a < b) {
      const uint64_t mid = (a + b) >> 1;
      if (w.piece_base[mid] < lo) a = mid + 1; else b = mid;
    }
    for (uint64_t f = a + threadIdx.x; f <= g.nfiles; f += blockDim.x) {
      const uint32_t sb = w.piece_base[f];
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

struct WLayout {
  size_t hdr, piece_base, list_base, ftile, ftile_l, piece_file, order, spec_n, spec, jin,
      jn, jm, jexit, jcut, first_bad, count, ctile, sdone, bad, runs, claim, total;
  uint64_t npmax, nlist, nftiles, nctiles;
  uint32_t P, fullcap;
};

WLayout make_wlayout(const seqcdc_params_t *p, uint64_t total, uint64_t nfiles, uint32_t P) {
  WLayout l{};
  l.P = P;
  l.fullcap = list_cap(P, (uint32_t)p->min_size);
  l.npmax = total / P + nfiles + 1;
  // Per file: (n / P) full lists plus one for the tail; summed over files at
  // most total / min_size + 3 (total / P + nfiles).
  l.nlist = total / p->min_size + 3 * l.npmax;
  l.nftiles = (nfiles + kFileTile - 1) / kFileTile;
  if (l.nftiles == 0) l.nftiles = 1;
  l.nctiles = (l.npmax + 1 + kPieceTile - 1) / kPieceTile;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  l.hdr = take(sizeof(WalkHeader));
  l.piece_base = take((nfiles + 1) * 4);
  l.list_base = take((nfiles + 1) * 8);
  l.ftile = take(l.nftiles * 4);
  l.ftile_l = take(l.nftiles * 8);
  l.piece_file = take(l.npmax * 4);
  l.order = take(l.npmax * 4);
  l.spec_n = take(l.npmax * 4);
  l.spec = take(l.nlist * 4);
  l.jin = take(l.npmax * 4);
  l.jn = take(l.npmax * 4);
  l.jm = take(l.npmax * 4);
  l.jexit = take(l.npmax * 4);
  l.jcut = take(l.nlist * 4);
  l.first_bad = take((nfiles + 1) * 4);
  l.count = take(l.npmax * 4);
  l.ctile = take(l.nctiles * 4);
  l.sdone = take(l.npmax * 4);
  l.bad = take(l.npmax * 4);
  l.runs = take(l.npmax * 4);
  l.claim = take(l.npmax * 4);
  l.total = o;
  return l;
}

WPtrs wptrs(void *d_ws, const WLayout &l) {
  char *b = static_cast<char *>(d_ws);
  WPtrs w;
  w.hdr = reinterpret_cast<WalkHeader *>(b + l.hdr);
  w.piece_base = reinterpret_cast<uint32_t *>(b + l.piece_base);
  w.list_base = reinterpret_cast<uint64_t *>(b + l.list_base);
  w.ftile = reinterpret_cast<uint32_t *>(b + l.ftile);
  w.ftile_l = reinterpret_cast<uint64_t *>(b + l.ftile_l);
  w.piece_file = reinterpret_cast<uint32_t *>(b + l.piece_file);
  w.order = reinterpret_cast<uint32_t *>(b + l.order);
  w.spec_n = reinterpret_cast<uint32_t *>(b + l.spec_n);
  w.spec = reinterpret_cast<uint32_t *>(b + l.spec);
  w.jin = reinterpret_cast<uint32_t *>(b + l.jin);
  w.jn = reinterpret_cast<uint32_t *>(b + l.jn);
  w.jm = reinterpret_cast<uint32_t *>(b + l.jm);
  w.jexit = reinterpret_cast<uint32_t *>(b + l.jexit);
  w.jcut = reinterpret_cast<uint32_t *>(b + l.jcut);
  w.first_bad = reinterpret_cast<uint32_t *>(b + l.first_bad);
  w.count = reinterpret_cast<uint32_t *>(b + l.count);
  w.ctile = reinterpret_cast<uint32_t *>(b + l.ctile);
  w.sdone = reinterpret_cast<uint32_t *>(b + l.sdone);
  w.bad = reinterpret_cast<uint32_t *>(b + l.bad);
  w.runs = reinterpret_cast<uint32_t *>(b + l.runs);
  w.claim = reinterpret_cast<uint32_t *>(b + l.claim);
  return w;
}

}  // namespace

namespace seqcdc_walk {

uint32_t pick_piece(const seqcdc_params_t *p, const seqcdc_tuning_t *t) {
  // Default: chains started at a piece start need about 25 chunks on
  // average, and up to ~120, to meet the true chain; chunks (and skips) grow
  // with min_size, so pieces do too.  Measured on a 10,000-file batch:
  // 768 KiB is best at min 1 KiB and 4 KiB, 3 MiB (384 x min) at min 8 KiB.
  uint64_t P = kDefaultPiece;
  if (p && p->min_size > 4096u) P = 384u * p->min_size;
  if (t && t->piece_bytes) P = t->piece_bytes;
  const uint64_t floor = p ? 4u * p->max_size : 0u;
  if (P < floor) P = floor;
  P = (P + 65535u) & ~(uint64_t)65535u;
  if (P > (64u << 20)) P = 64u << 20;
  return (uint32_t)P;
}

size_t workspace_bytes(const seqcdc_params_t *p, uint64_t total, uint64_t nfiles,
                       uint32_t piece) {
  return make_wlayout(p, total, nfiles, piece).total;
}

int run(const seqcdc_params_t *p, const uint8_t *d_data, uint64_t total,
        const uint64_t *d_offsets, uint64_t nfiles, uint64_t *d_cuts, uint64_t cap,
        uint64_t *d_cut_offsets, uint64_t *d_count, void *d_ws, size_t ws_bytes,
        uint32_t piece, int sms, bool host_data, void *stream, void *prof_begin,
        void *prof_end) {
  const WLayout l = make_wlayout(p, total, nfiles, piece);
  if (l.npmax >= 0xffffffffull || nfiles >= 0xffffffffull) return SEQCDC_ERANGE;
  if (ws_bytes < l.total) return SEQCDC_ECAPACITY;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const WPtrs w = wptrs(d_ws, l);
  const WGeom g{d_data, total, d_offsets, nfiles, l.P, l.fullcap, host_data ? 1u : 0u};
  const DevParams dp{p->mode, p->seq_length, p->skip_trigger, p->skip_size,
                     (uint32_t)p->min_size, (uint32_t)p->max_size};
  wplan_tiles_kernel<<<(unsigned)l.nftiles, 256, 0, st>>>(g, dp, w);
  wplan_scan_kernel<<<(unsigned)l.nftiles, 256, 0, st>>>(g, dp, w, l.nftiles);
  wfill_kernel<<<(unsigned)((l.npmax + 255) / 256), 256, 0, st>>>(g, w);
  // Persistent walk grids: up to 16 blocks of four warps per SM; warps take
  // pieces from a queue, so blocks that do not fit only find it empty.
  const uint64_t want = (l.npmax + 3) / 4;
  const uint64_t most = 16u * (uint64_t)sms;
  const unsigned wgrid = (unsigned)(want < most ? want : most);
  if (prof_begin) record_event(static_cast<cudaEvent_t>(prof_begin), st);
  const int variant = (dp.mode ? 2 : 0) + (dp.R == 5u ? 1 : 0);
  // Input in host memory: the walks load each half window only when the
  // scan reaches it (the bytes that cross to the GPU bound the walk there).
  void (*const walk_fns[8])(WGeom, DevParams, WPtrs) = {
      walk_kernel<0, false, false>, walk_kernel<0, true, false>,
      walk_kernel<1, false, false>, walk_kernel<1, true, false>,
      walk_kernel<0, false, true>,  walk_kernel<0, true, true>,
      walk_kernel<1, false, true>,  walk_kernel<1, true, true>};
  void (*const run_fns[4])(WGeom, DevParams, WPtrs, uint32_t) = {
      wrun_repair_kernel<0, false>, wrun_repair_kernel<0, true>, wrun_repair_kernel<1, false>,
      wrun_repair_kernel<1, true>};
  void (*const rep_fns[4])(WGeom, DevParams, WPtrs) = {
      wrepair_kernel<0, false>, wrepair_kernel<0, true>, wrepair_kernel<1, false>,
      wrepair_kernel<1, true>};
  walk_fns[variant + (host_data ? 4 : 0)]<<<wgrid, kWalkThreads, 0, st>>>(g, dp, w);
  if (prof_end) record_event(static_cast<cudaEvent_t>(prof_end), st);
  const uint64_t vb = (l.npmax + 255) / 256;
  const unsigned vgrid = (unsigned)(vb < 4096 ? vb : 4096);
  // Rounds of verify + parallel run repair (a persistent grid of warps takes
  // runs from the round's list), then the last verify for the sequential
  // repair of whatever is left.
  const uint64_t rwant = (l.npmax + 3) / 4;
  const uint64_t rmost = 2u * (uint64_t)sms;
  const unsigned rrgrid = (unsigned)(rwant < rmost ? (rwant ? rwant : 1) : rmost);
  for (uint32_t round = 0; round < kWalkRepairRounds; ++round) {
    wverify_kernel<<<vgrid, 256, 0, st>>>(g, dp, w, round);
    run_fns[variant]<<<rrgrid, kWalkThreads, 0, st>>>(g, dp, w, round);
  }
  wverify_kernel<<<vgrid, 256, 0, st>>>(g, dp, w, kWalkRepairRounds);
  const uint64_t rb = (nfiles + 3) / 4;
  const uint64_t rcap = 4u * (uint64_t)sms;
  rep_fns[variant]<<<(unsigned)(rb < rcap ? (rb ? rb : 1) : rcap), kWalkThreads, 0, st>>>(g, dp, w);
  wcount_kernel<<<(unsigned)l.nctiles, kPieceTile, 0, st>>>(g, dp, w);
  wemit_kernel<<<(unsigned)l.nctiles, kEmitThreads, 0, st>>>(g, dp, w, d_cuts, cap,
                                                             d_cut_offsets, d_count);
  return cudaGetLastError() == cudaSuccess ? SEQCDC_OK : SEQCDC_ECUDA;
}

}  // namespace seqcdc_walk
