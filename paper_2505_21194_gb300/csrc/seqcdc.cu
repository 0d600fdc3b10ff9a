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
// The scan region of Sec. III.D is evaluated here as bitmaps: T[j] marks a
// target-order pair (b[j-1], b[j]), O[j] an opposing pair, and
// E[j] = T[j] & T[j-1] & ... & T[j-SeqLength+2] marks the last byte of a
// boundary run -- the AND of SeqLength-1 shifted comparison masks of
// Sec. III.D.  A region starting at byte i ends at the first E bit at or after
// i + SeqLength - 1 (a cut after it) or at the SkipTrigger-th O bit after i
// (a skip), whichever comes first.
//
// Parallel structure (not in the paper, which scans sequentially):
//   plan kernels   split every file into segments of L bytes (items).
//   segment kernel one thread block per item.  It stages the item's bytes
//                  plus max_size bytes of look-ahead, builds the E and O
//                  bitmaps in shared memory (SWAR byte compares, 16 bytes per
//                  thread per step), and then walks the chunk chain from EVERY
//                  position a chunk of this file could start at inside the
//                  item's first max_size bytes (each natural cut is E+1), with
//                  chains that reach a common cut merged through a shared-memory
//                  hash.  The result is a table entry -> exit (first cut at or
//                  after the item end) and the set of distinct exits.  The
//                  table is published; the block then finds its true entry by
//                  a bounded look-back over its predecessors' tables (a
//                  single-valued exit set settles it at once) and emits its
//                  true cuts from shared memory.
//   compact        exclusive scan of per-item cut counts, then a copy into the
//                  caller's CSR output.
// The output equals a sequential scan's exactly: every cut of an item is
// produced by the same state machine from a proven true chunk start.

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "seqcdc.h"

namespace {

// ---------------------------------------------------------------------------
// Limits and layout constants.
// ---------------------------------------------------------------------------
constexpr int kMaxEntries = 512;    // entry candidates tabulated per item
constexpr int kMaxNodes = 1024;     // distinct cut positions per item walk
constexpr int kHashSlots = 2048;    // open-addressing slots (power of two)
constexpr int kMaxImage = 32;       // distinct exits published per item (one per lane)
constexpr int kFileTile = 1024;     // files per plan block
constexpr int kItemTile = 256;      // items per compaction block
constexpr uint32_t kMaxSeqLength = 16;
constexpr uint64_t kMaxMaxSize = 262144;
constexpr int64_t kLookBackDepth = 6;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on any device wait

// Item state bits.
constexpr uint32_t F_TABLE = 1u;     // exit set (and maybe table) published
constexpr uint32_t F_SINGLE = 2u;    // exit set has exactly one element
constexpr uint32_t F_NOTABLE = 4u;   // no usable table (too many exits)
constexpr uint32_t F_RESOLVED = 8u;  // entry chosen, cuts and exit published
constexpr uint32_t F_ABNORMAL = 16u; // no walk from all entries was possible
constexpr uint32_t F_UNRESOLVED = 32u;  // look-back could not choose an entry

constexpr uint16_t kNil = 0xFFFFu;
constexpr uint32_t kInvalidPos = 0xFFFFFFFFu;

struct DevParams {
  uint32_t mode;
  uint32_t R;   // seq_length
  uint32_t T;   // skip_trigger (0 = never)
  uint32_t S;   // skip_size
  uint32_t mn;  // min_size
  uint32_t mx;  // max_size
};

// Workspace header (first 256 bytes of the workspace).
struct WsHeader {
  uint32_t status;
  uint32_t ticket;
  uint32_t nitems;
  uint32_t pad[61];
};

struct Layout {
  size_t hdr, seg_base, ftile, state, incl, entry, first_bad, count, img_n,
      img, tab_n, tab, slot, itile, total;
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
};

__host__ __device__ inline uint64_t file_start(const Geom &g, uint64_t f) {
  return g.offsets ? g.offsets[f] : 0;
}
__host__ __device__ inline uint64_t file_size(const Geom &g, uint64_t f) {
  return g.offsets ? g.offsets[f + 1] - g.offsets[f] : g.total;
}

struct WsPtrs {
  WsHeader *hdr;
  uint32_t *seg_base;   // nfiles + 1
  uint32_t *ftile;      // per plan tile
  uint32_t *state;      // per item
  uint64_t *incl;       // per item: exit from `entry` (file-relative)
  uint64_t *entry;      // per item: entry the item's cuts were computed from
  uint32_t *first_bad;  // per file: first inconsistent item (verify pass)
  uint32_t *count;      // per item: true cuts emitted
  uint32_t *img_n;      // per item
  uint64_t *img;        // per item x kMaxImage (file-relative)
  uint32_t *tab_n;      // per item
  uint64_t *tab;        // per item x kMaxEntries
  uint64_t *slot;       // per item x slot_cap (file-relative cuts)
  uint32_t *itile;      // per compaction tile
  uint32_t slot_cap;
};

// ---------------------------------------------------------------------------
// Small device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait until (*flag & mask) != 0, at most kWaitNs.  Returns the flag value, or
// 0 after recording SEQCDC_ETIMEOUT in the workspace status.
__device__ uint32_t wait_any(const uint32_t *flag, uint32_t mask, WsHeader *hdr) {
  uint64_t t0 = global_ns();
  uint32_t backoff = 32;
  for (uint64_t it = 0; it < (1ull << 32); ++it) {
    uint32_t v = ld_acquire(flag);
    if (v & mask) return v;
    if (global_ns() - t0 > kWaitNs) break;
    __nanosleep(backoff);
    if (backoff < 1024) backoff <<= 1;
  }
  atomicExch(&hdr->status, (uint32_t)SEQCDC_ETIMEOUT);
  return 0;
}

// Per-byte "a > b" for four unsigned bytes; the answer is in bit 7 of each
// byte, the other bits are garbage.  Low seven bits are compared with a
// borrow-free subtraction ((a | 0x80) - (b & 0x7f) - 1 stays within 0..0xff),
// the high bits decide when they differ.
__device__ __forceinline__ uint32_t gt_hi(uint32_t a, uint32_t b) {
  uint32_t z = (a | 0x80808080u) - (b & 0x7f7f7f7fu) - 0x01010101u;
  return (a & ~b) | (~(a ^ b) & z);
}

// Gather bit 7 of each byte into bits 0..3 (byte k -> bit k).
__device__ __forceinline__ uint32_t pack4(uint32_t m) {
  return ((m & 0x80808080u) * 0x00204081u) >> 28;
}

// Position (0..31) of the k-th set bit (k >= 1, k <= popc(x)).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t x, uint32_t k) {
  uint32_t pos = 0;
  uint32_t c = __popc(x & 0xffffu);
  if (k > c) { k -= c; x >>= 16; pos += 16; }
  c = __popc(x & 0xffu);
  if (k > c) { k -= c; x >>= 8; pos += 8; }
  c = __popc(x & 0xfu);
  if (k > c) { k -= c; x >>= 4; pos += 4; }
  c = __popc(x & 0x3u);
  if (k > c) { k -= c; x >>= 2; pos += 2; }
  c = x & 1u;
  if (k > c) { pos += 1; }
  return pos;
}

// Target / opposing bit masks (16 positions) for the 16 bytes in v, given the
// byte before them.  Bit t of the result refers to the pair
// (byte t-1, byte t) of this group.
__device__ __forceinline__ void classify16(uint32_t prev_byte, uint4 v,
                                           uint32_t mode, uint32_t &T16,
                                           uint32_t &O16) {
  uint32_t x0 = v.x, x1 = v.y, x2 = v.z, x3 = v.w;
  uint32_t y0 = (x0 << 8) | (prev_byte & 0xffu);
  uint32_t y1 = __funnelshift_l(x0, x1, 8);
  uint32_t y2 = __funnelshift_l(x1, x2, 8);
  uint32_t y3 = __funnelshift_l(x2, x3, 8);
  uint32_t up = pack4(gt_hi(x0, y0)) | (pack4(gt_hi(x1, y1)) << 4) |
                (pack4(gt_hi(x2, y2)) << 8) | (pack4(gt_hi(x3, y3)) << 12);
  uint32_t dn = pack4(gt_hi(y0, x0)) | (pack4(gt_hi(y1, x1)) << 4) |
                (pack4(gt_hi(y2, x2)) << 8) | (pack4(gt_hi(y3, x3)) << 12);
  T16 = mode == 0 ? up : dn;
  O16 = mode == 0 ? dn : up;
}

// 16 input bytes starting at global byte index gi (16-aligned); bytes outside
// [0, total) read as zero.
__device__ __forceinline__ uint4 load16(const uint8_t *data, int64_t gi,
                                        uint64_t total) {
  if (gi >= 0 && (uint64_t)gi + 16 <= total) {
    return __ldg(reinterpret_cast<const uint4 *>(data + gi));
  }
  uint32_t w[4] = {0, 0, 0, 0};
  for (int t = 0; t < 16; ++t) {
    int64_t a = gi + t;
    if (a >= 0 && (uint64_t)a < total) w[t >> 2] |= (uint32_t)data[a] << (8 * (t & 3));
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// ---------------------------------------------------------------------------
// Shared-memory view of one item's bitmaps.  Positions are relative to the
// window base B (file-relative): rel = pos - B.  Word w covers rel 32w..32w+31.
// ---------------------------------------------------------------------------
struct Bits {
  const uint32_t *E;
  const uint32_t *O;
};

// Event of one scan region starting at rel i (bytes i.. ; pairs i+1..).
// Returns the cut (rel, > 0) if a boundary run ends first, or sets *skip to
// the rel position of the trigger pair and returns 0, or returns 0 with
// *skip = kInvalidPos if neither happens before rel `limit`.
__device__ __forceinline__ uint32_t scan_region(const Bits &b,
                                                const DevParams &p, uint32_t i,
                                                uint32_t limit,
                                                uint32_t *skip) {
  const uint32_t o_start = i + 1;
  const uint32_t e_start = i + p.R - 1;
  uint32_t need = p.T;
  uint32_t w = o_start >> 5;
  const uint32_t w_end = (limit + 31) >> 5;
  for (; w < w_end; ++w) {
    const uint32_t base = w << 5;
    uint32_t ob = b.O[w];
    uint32_t eb = b.E[w];
    if (o_start > base) ob &= ~0u << (o_start - base);
    if (e_start > base) eb = (e_start - base >= 32) ? 0u : (eb & (~0u << (e_start - base)));
    if (limit - base < 32) {
      const uint32_t m = (1u << (limit - base)) - 1u;
      ob &= m;
      eb &= m;
    }
    if (need != 0) {
      const uint32_t pc = __popc(ob);
      if (pc >= need) {
        const uint32_t sb = nth_set_bit(ob, need);
        const uint32_t before = eb & ((1u << sb) - 1u);
        if (before) return base + (__ffs(before) - 1) + 1;
        *skip = base + sb;
        return 0;
      }
      need -= pc;
    }
    if (eb) return base + (__ffs(eb) - 1) + 1;
  }
  *skip = kInvalidPos;
  return 0;
}

// One chunk: from chunk start c (rel) return its end (rel).  `end_rel` is the
// rel position of the file end (a hard limit).
__device__ uint32_t chunk_step(const Bits &b, const DevParams &p, uint32_t c,
                               uint32_t end_rel) {
  const uint32_t limit = (end_rel - c > p.mx) ? c + p.mx : end_rel;
  uint32_t i = c + (p.mn > p.R ? p.mn - p.R : 0u);
  while (i + 1 < limit) {
    uint32_t skip;
    const uint32_t cut = scan_region(b, p, i, limit, &skip);
    if (cut) return cut;
    if (skip == kInvalidPos) break;
    i = skip + 1 + p.S;
  }
  return limit;
}

__device__ __forceinline__ uint32_t hash_pos(uint32_t x) {
  return (x * 2654435761u) >> (32 - 11);  // kHashSlots = 2048
}

// Exclusive block scan of one value per thread (blockDim <= 1024).
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *scratch,
                                    uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  uint32_t x = v;
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < nwarps ? scratch[lane] : 0u;
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
      if (lane >= d) s += y;
    }
    if (lane < nwarps) scratch[lane] = s;
  }
  __syncthreads();
  const uint32_t warp_off = warp ? scratch[warp - 1] : 0u;
  *total = scratch[nwarps - 1];
  __syncthreads();
  return warp_off + x - v;
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
    const uint64_t n = file_size(g, f);
    sum += (uint32_t)((n + g.L - 1) / g.L);
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
  // Prefix of all previous tiles.
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
    uint32_t v = 0;
    if (f < g.nfiles && f < f0 + kFileTile) {
      const uint64_t n = file_size(g, f);
      v = (uint32_t)((n + g.L - 1) / g.L);
    }
    uint32_t tot;
    const uint32_t ex = block_excl_scan(v, scratch, &tot);
    if (f < g.nfiles && f < f0 + kFileTile) ws.seg_base[f] = running + ex;
    running += tot;
  }
  if (blockIdx.x == nftiles - 1 && threadIdx.x == 0) {
    ws.seg_base[g.nfiles] = running;
    ws.hdr->nitems = running;
    ws.hdr->ticket = 0;
    ws.hdr->status = 0;
  }
  // Reset per-item state and per-file repair marks.
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
// Segment kernel.
// ---------------------------------------------------------------------------
struct SegShared {
  uint32_t item, file, seg, nitems, first_item;
  int64_t B;          // window base (file-relative); global index of rel 0 is 16-aligned
  uint64_t p_s, q_s, n_f, gbase;
  uint32_t W;         // bitmap words
  uint32_t K;         // entries
  uint32_t nnodes, nact, nnew, abnormal, rounds, nimg;
  uint32_t scratch[32];
  uint64_t true_entry;
  uint32_t resolved;
};

// Pointers into the dynamic shared memory of one item.
struct SegSmem {
  uint32_t *E, *O;
  uint32_t *node_pos;     // kMaxNodes
  uint16_t *node_next;    // kMaxNodes
  uint16_t *hslot;        // kHashSlots
  uint16_t *act, *act2;   // kMaxNodes each
  uint64_t *img_local;    // kMaxImage
  uint16_t *img_of_node;  // kMaxNodes
};

__device__ __forceinline__ SegSmem carve(unsigned char *raw, uint32_t W) {
  SegSmem m;
  m.E = reinterpret_cast<uint32_t *>(raw);
  m.O = m.E + W;
  m.node_pos = m.O + W;
  m.node_next = reinterpret_cast<uint16_t *>(m.node_pos + kMaxNodes);
  m.hslot = m.node_next + kMaxNodes;
  m.act = m.hslot + kHashSlots;
  m.act2 = m.act + kMaxNodes;
  m.img_local = reinterpret_cast<uint64_t *>(m.act2 + kMaxNodes);
  m.img_of_node = reinterpret_cast<uint16_t *>(m.img_local + kMaxImage);
  return m;
}

__device__ __forceinline__ uint32_t find_file(const uint32_t *seg_base,
                                              uint64_t nfiles, uint32_t item) {
  // largest f < nfiles with seg_base[f] <= item (then seg_base[f+1] > item)
  uint64_t lo = 0, hi = nfiles;
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (seg_base[mid] <= item) lo = mid; else hi = mid;
  }
  return (uint32_t)lo;
}

// Geometry of item (file, seg); thread 0 only.
__device__ void seg_setup(SegShared &sh, const Geom &g, const DevParams &p,
                          uint32_t item, uint32_t file, uint32_t seg,
                          uint32_t first_item) {
  sh.item = item;
  sh.file = file;
  sh.seg = seg;
  sh.first_item = first_item;
  sh.n_f = file_size(g, file);
  sh.gbase = file_start(g, file);
  sh.p_s = (uint64_t)seg * g.L;
  sh.q_s = min(sh.p_s + g.L, sh.n_f);
  const uint64_t w1 = min(sh.q_s + p.mx, sh.n_f);
  // Window base: 32 bytes before the item, rounded down so that its global
  // byte index is 16-aligned.
  int64_t gb = (int64_t)(sh.gbase + sh.p_s) - 32;
  gb = gb >= 0 ? (gb & ~(int64_t)15) : -(((-gb) + 15) & ~(int64_t)15);
  sh.B = gb - (int64_t)sh.gbase;
  sh.W = (uint32_t)(((int64_t)w1 - sh.B + 31) >> 5);
  sh.abnormal = 0;
  sh.nnodes = 0;
  sh.K = 0;
  sh.nimg = 0;
  sh.resolved = 0;
}

// E and O bitmaps of the window [B, B + 32 W), 16 positions per lane step.
__device__ void seg_bitmaps(const SegShared &sh, const Geom &g,
                            const DevParams &p, const SegSmem &m) {
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const uint32_t W = sh.W;
  const int64_t gwin = (int64_t)sh.gbase + sh.B;  // global byte index of rel 0
  uint16_t *E16 = reinterpret_cast<uint16_t *>(m.E);
  uint16_t *O16 = reinterpret_cast<uint16_t *>(m.O);
  const uint32_t H = 2 * W;  // 16-byte groups
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
  uint32_t per = (H + nwarps - 1) / nwarps;
  per = (per + 31) & ~31u;
  const uint32_t h0 = warp * per;
  const uint32_t h1 = min(h0 + per, H);
  uint32_t carry_byte = 0, carry_T = 0;
  if (h0 < h1 && h0 > 0) {
    // T bits of the 16 positions before this warp's first group (only the top
    // SeqLength-2 of them matter, so the unknown byte before them is moot).
    const uint4 pv = load16(g.data, gwin + 16 * (int64_t)(h0 - 1), g.total);
    uint32_t t16, o16;
    classify16(0, pv, p.mode, t16, o16);
    carry_T = t16;
    carry_byte = pv.w >> 24;
  }
  for (uint32_t hb = h0; hb < h1; hb += 32) {
    const uint32_t h = hb + lane;
    const bool live = h < h1;
    const uint4 v = live ? load16(g.data, gwin + 16 * (int64_t)h, g.total)
                         : make_uint4(0, 0, 0, 0);
    uint32_t pb = __shfl_up_sync(0xffffffffu, v.w >> 24, 1);
    if (lane == 0) pb = carry_byte;
    uint32_t t16, o16;
    classify16(pb, v, p.mode, t16, o16);
    uint32_t pt = __shfl_up_sync(0xffffffffu, t16, 1);
    if (lane == 0) pt = carry_T;
    // E at group position t needs T at t, t-1, ..., t-(R-2): the previous
    // group's T bits sit below this group's in a 32-bit window.
    const uint32_t tw = (t16 << 16) | (pt & 0xffffu);
    uint32_t ew = tw;
    for (uint32_t k = 1; k + 1 < p.R; ++k) ew &= tw << k;
    if (live) {
      E16[h] = (uint16_t)(ew >> 16);
      O16[h] = (uint16_t)o16;
    }
    carry_byte = __shfl_sync(0xffffffffu, v.w >> 24, 31);
    carry_T = __shfl_sync(0xffffffffu, t16, 31);
  }
}

// Phases 2-4: entry candidates, walk of every entry's chain with merging,
// exits and the entry -> exit table, published to the workspace.  All threads.
__device__ void seg_walk_publish(SegShared &sh, const DevParams &p,
                                 const SegSmem &m, const WsPtrs &ws) {
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int64_t B = sh.B;
  const uint64_t n_f = sh.n_f, p_s = sh.p_s, q_s = sh.q_s;
  const uint32_t end_rel = (uint32_t)((int64_t)n_f - B);
  const uint32_t q_rel = (uint32_t)((int64_t)q_s - B);
  const uint32_t ps_rel = (uint32_t)((int64_t)p_s - B);
  const Bits bits{m.E, m.O};
  const uint32_t item = sh.item;

  // Entry candidates.  Item 0 of a file starts at the file start; any other
  // item may be entered at every natural cut x = e + 1 (E[e] set) with
  // p_s <= x < p_s + max_size.
  if (sh.seg == 0) {
    if (tid == 0) {
      m.node_pos[0] = ps_rel;
      sh.K = 1;
    }
  } else {
    const uint64_t xe = min(p_s + (uint64_t)p.mx, n_f);  // entries x < xe
    const uint32_t lo = ps_rel - 1;                      // e >= lo
    const uint32_t hi = (uint32_t)((int64_t)xe - B) - 1; // e < hi
    const uint32_t wlo = lo >> 5, whi = (hi + 31) >> 5;
    const uint32_t nw = whi - wlo;
    const uint32_t per = (nw + nthreads - 1) / nthreads;
    const uint32_t a = wlo + tid * per, z = min(a + per, whi);
    uint32_t cnt = 0;
    for (uint32_t w = a; w < z; ++w) {
      uint32_t v = m.E[w];
      const uint32_t base = w << 5;
      if (lo > base) v &= ~0u << (lo - base);
      if (hi - base < 32) v &= (1u << (hi - base)) - 1u;
      cnt += __popc(v);
    }
    uint32_t K;
    const uint32_t off = block_excl_scan(cnt, sh.scratch, &K);
    if (K == 0 || K > (uint32_t)kMaxEntries) {
      if (tid == 0) sh.abnormal = 1;
    } else {
      uint32_t o = off;
      for (uint32_t w = a; w < z; ++w) {
        uint32_t v = m.E[w];
        const uint32_t base = w << 5;
        if (lo > base) v &= ~0u << (lo - base);
        if (hi - base < 32) v &= (1u << (hi - base)) - 1u;
        while (v) {
          const uint32_t bpos = __ffs(v) - 1;
          v &= v - 1;
          m.node_pos[o++] = base + bpos + 1;
        }
      }
      if (tid == 0) sh.K = K;
    }
  }
  __syncthreads();

  // Walk every entry's chunk chain to its exit (first cut >= q_s), merging
  // chains that reach a common cut.  Nodes are distinct cut positions.
  if (!sh.abnormal) {
    const uint32_t K = sh.K;
    for (int i = tid; i < kHashSlots; i += nthreads) m.hslot[i] = kNil;
    for (int i = tid; i < kMaxNodes; i += nthreads) m.node_next[i] = kNil;
    if (tid == 0) {
      sh.nnodes = K;
      sh.nact = 0;
      sh.nnew = 0;
      sh.rounds = 0;
    }
    __syncthreads();
    for (uint32_t k = tid; k < K; k += nthreads) {
      const uint32_t x = m.node_pos[k];
      uint32_t slot = hash_pos(x);
      while (atomicCAS(&m.hslot[slot], kNil, (uint16_t)k) != kNil)
        slot = (slot + 1) & (kHashSlots - 1);
      if (x < q_rel) m.act[atomicAdd(&sh.nact, 1u)] = (uint16_t)k;
    }
    __syncthreads();
    uint16_t *cur_act = m.act, *nxt_act = m.act2;
    while (true) {
      const uint32_t nact = sh.nact;
      if (nact == 0 || sh.abnormal) break;
      for (uint32_t t = tid; t < nact; t += nthreads) {
        const uint16_t h = cur_act[t];
        const uint32_t y = chunk_step(bits, p, m.node_pos[h], end_rel);
        uint32_t slot = hash_pos(y);
        uint16_t id = kNil;
        bool created = false;
        for (int probe = 0; probe < kHashSlots; ++probe) {
          uint16_t cur = *((volatile uint16_t *)&m.hslot[slot]);
          if (cur == kNil) {
            const uint32_t nid = atomicAdd(&sh.nnodes, 1u);
            if (nid >= (uint32_t)kMaxNodes) {
              sh.abnormal = 1;
              break;
            }
            m.node_pos[nid] = y;
            m.node_next[nid] = kNil;
            __threadfence_block();
            const uint16_t prev = atomicCAS(&m.hslot[slot], kNil, (uint16_t)nid);
            if (prev == kNil) {
              id = (uint16_t)nid;
              created = true;
              break;
            }
            m.node_pos[nid] = kInvalidPos;  // lost the slot; the winner may match
            cur = prev;
          }
          if (*((volatile uint32_t *)&m.node_pos[cur]) == y) {
            id = cur;
            break;
          }
          slot = (slot + 1) & (kHashSlots - 1);
        }
        m.node_next[h] = id;
        if (created && y < q_rel) nxt_act[atomicAdd(&sh.nnew, 1u)] = id;
      }
      __syncthreads();
      if (tid == 0) {
        sh.nact = sh.nnew;
        sh.nnew = 0;
        sh.rounds++;
      }
      uint16_t *tmp = cur_act;
      cur_act = nxt_act;
      nxt_act = tmp;
      __syncthreads();
    }
  }
  __syncthreads();

  // Exits (terminal nodes) and, by pointer jumping, each entry's exit and hop
  // count.  Publish the exit set and, when it has several elements, the table.
  if (!sh.abnormal) {
    const uint32_t nn = min(sh.nnodes, (uint32_t)kMaxNodes);
    uint16_t *jmp = m.hslot;               // reuse the hash (kHashSlots >= 2*kMaxNodes)
    uint16_t *cnt = m.hslot + kMaxNodes;
    for (uint32_t n = tid; n < nn; n += nthreads) {
      const bool valid = m.node_pos[n] != kInvalidPos;
      const uint16_t nx = m.node_next[n];
      if (valid && nx == kNil) {
        const uint32_t idx = atomicAdd(&sh.nimg, 1u);
        if (idx < (uint32_t)kMaxImage) m.img_local[idx] = (uint64_t)(B + (int64_t)m.node_pos[n]);
        m.img_of_node[n] = (uint16_t)idx;
      }
      jmp[n] = (nx == kNil) ? (uint16_t)n : nx;
      cnt[n] = (nx == kNil) ? 0 : 1;
    }
    __syncthreads();
    // A path can pass through several merged chains, so its length is bounded
    // by the node count, not by the number of rounds.
    for (uint32_t r = 1; r < 2 * nn; r <<= 1) {
      for (uint32_t n = tid; n < nn; n += nthreads) {
        const uint16_t j = jmp[n];
        m.act[n] = jmp[j];
        m.act2[n] = cnt[n] + cnt[j];
      }
      __syncthreads();
      for (uint32_t n = tid; n < nn; n += nthreads) {
        jmp[n] = m.act[n];
        cnt[n] = m.act2[n];
      }
      __syncthreads();
    }
    const uint32_t nimg = sh.nimg;
    const bool notable = nimg > (uint32_t)kMaxImage;
    if (!notable) {
      for (uint32_t k = tid; k < nimg; k += nthreads)
        ws.img[(uint64_t)item * kMaxImage + k] = m.img_local[k];
      if (nimg > 1) {
        for (uint32_t k = tid; k < sh.K; k += nthreads) {
          const uint16_t ex = jmp[k];
          const uint64_t ent = (uint64_t)(m.node_pos[k] - ps_rel);
          ws.tab[(uint64_t)item * kMaxEntries + k] =
              ent | ((uint64_t)m.img_of_node[ex] << 32) | ((uint64_t)cnt[k] << 40);
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      ws.img_n[item] = nimg;
      ws.tab_n[item] = sh.K;
      __threadfence();
      atomicOr(&ws.state[item], F_TABLE | (nimg == 1 ? F_SINGLE : 0u) |
                                    (notable ? F_NOTABLE : 0u));
    }
  } else if (tid == 0) {
    __threadfence();
    atomicOr(&ws.state[item], F_ABNORMAL);
  }
}

// Exit of item j for entry position x (file-relative), from j's table.
// Returns false if x is not one of j's entries.
__device__ bool table_lookup(const WsPtrs &ws, uint32_t j, uint64_t pj,
                             uint64_t x, uint64_t *out) {
  if (x < pj) return false;
  const uint64_t want = x - pj;
  const uint64_t *tb = ws.tab + (uint64_t)j * kMaxEntries;
  uint32_t lo = 0, hi = __ldcg(&ws.tab_n[j]);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint64_t v = __ldcg(&tb[mid]);
    const uint64_t ent = v & 0xffffffffull;
    if (ent == want) {
      *out = __ldcg(&ws.img[(uint64_t)j * kMaxImage + ((v >> 32) & 0xff)]);
      return true;
    }
    if (ent < want) lo = mid + 1; else hi = mid;
  }
  return false;
}

// Speculative entry of a non-first item by look-back over the predecessors'
// published exit sets and tables (warp 0).  The candidates for this item's
// entry are the exits of item s-1 over its entries; when there are several,
// the exits of s-2 are pushed through s-1's table, and so on, up to
// kLookBackDepth items.  The result assumes each predecessor was entered at
// one of its tabulated entries; the verify pass checks that afterwards.
// Waits only for predecessors' tables, which depend on nothing else.
__device__ void seg_lookback(SegShared &sh, const Geom &g, const WsPtrs &ws) {
  const int lane = threadIdx.x & 31;
  const uint32_t item = sh.item;
  const uint32_t first_item = sh.first_item;
  bool ok = false;
  uint64_t x = 0;
  for (uint32_t depth = 1; depth <= (uint32_t)kLookBackDepth; ++depth) {
    const uint32_t k = item - depth;  // k >= first_item (item 0 is single)
    uint32_t st = 0;
    if (lane == 0) st = wait_any(&ws.state[k], F_TABLE | F_ABNORMAL, ws.hdr);
    st = __shfl_sync(0xffffffffu, st, 0);
    if (st == 0) break;
    st = ld_acquire(&ws.state[k]);  // every lane acquires before reading k's data
    if (st & (F_ABNORMAL | F_NOTABLE)) break;
    const uint32_t nimg = __ldcg(&ws.img_n[k]);
    // Each lane pushes one of k's exits through the tables of k+1 .. item-1.
    bool have = lane < (int)nimg;
    bool fail = false;
    uint64_t y = have ? __ldcg(&ws.img[(uint64_t)k * kMaxImage + lane]) : 0;
    for (uint32_t j = k + 1; j < item && have; ++j) {
      uint64_t z;
      if (table_lookup(ws, j, (uint64_t)(j - first_item) * g.L, y, &z)) y = z;
      else { fail = true; have = false; }
    }
    if (__any_sync(0xffffffffu, fail)) break;
    const uint64_t y0 = __shfl_sync(0xffffffffu, y, 0);
    const bool same = !(lane < (int)nimg) || y == y0;
    if (__all_sync(0xffffffffu, same)) {
      x = y0;
      ok = true;
      break;
    }
    if (k == first_item) break;
  }
  if (lane == 0) {
    sh.true_entry = x;
    sh.resolved = ok ? 1u : 0u;
  }
}

// Emission from entry x (file-relative): the cuts in (x, exit] into the
// item's slot, by following the walked nodes when x is a tabulated entry,
// else by stepping the chunker on the bitmaps.  Thread 0.
__device__ void seg_emit(SegShared &sh, const DevParams &p, const SegSmem &m,
                         const WsPtrs &ws, uint64_t x, bool use_nodes) {
  const int64_t B = sh.B;
  const Bits bits{m.E, m.O};
  const uint32_t end_rel = (uint32_t)((int64_t)sh.n_f - B);
  const uint32_t q_rel = (uint32_t)((int64_t)sh.q_s - B);
  const uint32_t item = sh.item;
  const uint32_t xr = (uint32_t)((int64_t)x - B);
  uint64_t *out = ws.slot + (uint64_t)item * ws.slot_cap;
  uint32_t nout = 0;
  uint64_t exit_pos = x;
  int node = -1;
  if (use_nodes) {
    uint32_t lo = 0, hi = sh.K;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      const uint32_t v = m.node_pos[mid];
      if (v == xr) { node = (int)mid; break; }
      if (v < xr) lo = mid + 1; else hi = mid;
    }
  }
  if (node >= 0) {
    uint32_t n = (uint32_t)node;
    while (m.node_next[n] != kNil && nout < ws.slot_cap) {
      n = m.node_next[n];
      out[nout++] = (uint64_t)(B + (int64_t)m.node_pos[n]);
    }
    exit_pos = (uint64_t)(B + (int64_t)m.node_pos[n]);
  } else {
    uint32_t c = xr;
    while (c < q_rel && nout < ws.slot_cap) {
      c = chunk_step(bits, p, c, end_rel);
      out[nout++] = (uint64_t)(B + (int64_t)c);
    }
    exit_pos = (uint64_t)(B + (int64_t)c);
  }
  ws.count[item] = nout;
  ws.incl[item] = exit_pos;
  ws.entry[item] = x;
  __threadfence();
  atomicOr(&ws.state[item], F_RESOLVED);
}

__global__ void __launch_bounds__(512)
segment_kernel(Geom g, DevParams p, WsPtrs ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SegShared sh;
  const int tid = threadIdx.x;
  if (tid == 0) {
    sh.item = atomicAdd(&ws.hdr->ticket, 1u);
    sh.nitems = ws.hdr->nitems;
  }
  __syncthreads();
  if (sh.item >= sh.nitems) return;
  if (tid == 0) {
    const uint32_t item = sh.item;
    const uint32_t f = find_file(ws.seg_base, g.nfiles, item);
    seg_setup(sh, g, p, item, f, item - ws.seg_base[f], ws.seg_base[f]);
  }
  __syncthreads();
  const SegSmem m = carve(smem_raw, sh.W);
  seg_bitmaps(sh, g, p, m);
  __syncthreads();
  seg_walk_publish(sh, p, m, ws);
  __syncthreads();
  if (sh.seg == 0) {
    if (tid == 0) {
      sh.true_entry = 0;
      sh.resolved = 1;
    }
  } else if (tid < 32) {
    seg_lookback(sh, g, ws);
  }
  __syncthreads();
  if (tid == 0) {
    if (sh.resolved) seg_emit(sh, p, m, ws, sh.true_entry, !sh.abnormal);
    else atomicOr(&ws.state[sh.item], F_UNRESOLVED);
  }
}

// Verify: item s of a file is consistent when it was resolved and its entry
// equals the exit its predecessor computed.  By induction from the file start
// (always a true entry), a file whose items are all consistent is exact.  The
// first inconsistent item of each file is recorded for the repair pass.
__global__ void verify_kernel(Geom g, WsPtrs ws) {
  const uint32_t nitems = ws.hdr->nitems;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nitems;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t f = find_file(ws.seg_base, g.nfiles, (uint32_t)i);
    const uint32_t s = (uint32_t)i - ws.seg_base[f];
    const uint32_t st = ws.state[i];
    bool ok = (st & F_RESOLVED) != 0;
    if (ok && s > 0) ok = ws.entry[i] == ws.incl[i - 1] && (ws.state[i - 1] & F_RESOLVED);
    if (!ok) atomicMin(&ws.first_bad[f], s);
  }
}

// Repair: one block per file with an inconsistent item.  From the first
// inconsistent item on, items are re-chunked from the true exit of their
// predecessor (bitmaps rebuilt from the input); an item whose recorded entry
// already equals that exit is kept.
__global__ void __launch_bounds__(512)
repair_kernel(Geom g, DevParams p, WsPtrs ws) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ SegShared sh;
  __shared__ uint32_t s_run;
  const int tid = threadIdx.x;
  for (uint64_t f = blockIdx.x; f < g.nfiles; f += gridDim.x) {
    const uint32_t fb = ws.first_bad[f];
    if (fb == 0xffffffffu) continue;
    const uint32_t base = ws.seg_base[f];
    const uint32_t nseg = ws.seg_base[f + 1] - base;
    uint64_t cur = ws.incl[base + fb - 1];  // fb >= 1: item 0 is always exact
    for (uint32_t s = fb; s < nseg; ++s) {
      const uint32_t item = base + s;
      if (tid == 0) {
        const uint32_t st = ws.state[item];
        s_run = !((st & F_RESOLVED) && ws.entry[item] == cur);
        if (s_run) seg_setup(sh, g, p, item, (uint32_t)f, s, base);
      }
      __syncthreads();
      if (s_run) {
        const SegSmem m = carve(smem_raw, sh.W);
        seg_bitmaps(sh, g, p, m);
        __syncthreads();
        if (tid == 0) seg_emit(sh, p, m, ws, cur, false);
      }
      __syncthreads();
      cur = *((volatile uint64_t *)&ws.incl[item]);
      __syncthreads();
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

__global__ void emit_kernel(Geom g, WsPtrs ws, uint64_t *d_cuts, uint64_t cap,
                            uint64_t *d_cut_offsets, uint64_t *d_count) {
  __shared__ uint32_t scratch[32];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t offs[kItemTile + 1];
  const uint32_t nitems = ws.hdr->nitems;
  const uint64_t lo = (uint64_t)blockIdx.x * kItemTile;
  // Prefix of all earlier tiles.
  uint64_t part = 0;
  for (uint64_t t = threadIdx.x; t < blockIdx.x; t += blockDim.x) part += ws.itile[t];
  for (int d = 16; d; d >>= 1) part += __shfl_down_sync(0xffffffffu, part, d);
  __shared__ uint64_t red64[32];
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
  // Copy: one warp per item.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int it = warp; it < kItemTile; it += blockDim.x >> 5) {
    const uint64_t item = lo + it;
    if (item >= nitems) break;
    const uint32_t n = ws.count[item];
    const uint64_t *src = ws.slot + item * ws.slot_cap;
    const uint64_t at = prefix + offs[it];
    if (at + n > cap) {  // cannot happen for a correct cut list; never write past cap
      if (lane == 0) atomicExch(&ws.hdr->status, (uint32_t)SEQCDC_ECAPACITY);
      continue;
    }
    uint64_t *dst = d_cuts + at;
    for (uint32_t j = lane; j < n; j += 32) dst[j] = src[j];
  }
  // CSR offsets of the files whose first item index falls in [lo, lo+tile).
  const uint64_t hi = lo + kItemTile;
  if (lo <= nitems) {
    // lower_bound(seg_base, lo) over [0, nfiles]
    uint64_t a = 0, b = g.nfiles + 1;
    while (a < b) {
      const uint64_t m = (a + b) >> 1;
      if (ws.seg_base[m] < lo) a = m + 1; else b = m;
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

uint32_t pick_segment(const seqcdc_params_t *p, const seqcdc_tuning_t *t) {
  uint32_t L = (t && t->segment_bytes) ? t->segment_bytes : 65536u;
  L = (L + 1023u) & ~1023u;
  if (L < 4096u) L = 4096u;
  if (L > (1u << 20)) L = 1u << 20;
  return L;
}

uint32_t pick_threads(const seqcdc_tuning_t *t) {
  uint32_t n = (t && t->block_threads) ? t->block_threads : 256u;
  if (n != 128u && n != 256u && n != 512u) n = 256u;
  return n;
}

size_t seg_smem_bytes(uint32_t L, uint64_t mx) {
  const uint64_t W = (L + mx + 64 + 31) / 32 + 2;
  return (size_t)(8 * W) + kMaxNodes * 4 + kMaxNodes * 2 + kHashSlots * 2 +
         kMaxNodes * 2 * 2 + kMaxImage * 8 + kMaxNodes * 2 + 64;
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
  l.tab_n = take(l.imax * 4);
  l.tab = take(l.imax * (size_t)kMaxEntries * 8);
  l.slot = take(l.imax * (size_t)l.slot_cap * 8);
  l.itile = take(l.nitiles * 4);
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
  w.tab_n = reinterpret_cast<uint32_t *>(b + l.tab_n);
  w.tab = reinterpret_cast<uint64_t *>(b + l.tab);
  w.slot = reinterpret_cast<uint64_t *>(b + l.slot);
  w.itile = reinterpret_cast<uint32_t *>(b + l.itile);
  w.slot_cap = l.slot_cap;
  return w;
}

thread_local cudaEvent_t g_prof_begin = nullptr;
thread_local cudaEvent_t g_prof_end = nullptr;

int run(const seqcdc_params_t *p, const uint8_t *d_data, uint64_t total,
        const uint64_t *d_offsets, uint64_t nfiles, uint64_t *d_cuts,
        uint64_t cap, uint64_t *d_cut_offsets, uint64_t *d_count, void *d_ws,
        size_t ws_bytes, const seqcdc_tuning_t *tuning, void *stream) {
  if (!params_ok(p)) return SEQCDC_EINVAL;
  if (!d_ws || ((uintptr_t)d_ws & 255u)) return SEQCDC_EINVAL;
  if (total > 0 && (!d_data || ((uintptr_t)d_data & 15u))) return SEQCDC_EINVAL;
  if (total > 0 && !d_cuts) return SEQCDC_EINVAL;
  const uint32_t L = pick_segment(p, tuning);
  const uint32_t threads = pick_threads(tuning);
  const Layout l = make_layout(p, total, nfiles, L);
  if (l.imax >= 0xffffffffull) return SEQCDC_ERANGE;
  if (ws_bytes < l.total) return SEQCDC_ECAPACITY;
  if (cap < total / p->min_size + nfiles) return SEQCDC_ECAPACITY;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const WsPtrs w = ws_ptrs(d_ws, l);
  Geom g{d_data, total, d_offsets, nfiles, L};
  DevParams dp{p->mode, p->seq_length, p->skip_trigger, p->skip_size,
               (uint32_t)p->min_size, (uint32_t)p->max_size};
  plan_tiles_kernel<<<(unsigned)l.nftiles, 256, 0, st>>>(g, w);
  plan_scan_kernel<<<(unsigned)l.nftiles, 256, 0, st>>>(g, w, l.nftiles, l.imax);
  const size_t smem = seg_smem_bytes(L, p->max_size);
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    if (cudaFuncSetAttribute(segment_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(repair_kernel,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return SEQCDC_ECUDA;
    configured = smem;
  }
  if (g_prof_begin) cudaEventRecord(g_prof_begin, st);
  segment_kernel<<<(unsigned)l.imax, threads, smem, st>>>(g, dp, w);
  if (g_prof_end) cudaEventRecord(g_prof_end, st);
  const uint64_t vblocks = (l.imax + 255) / 256;
  verify_kernel<<<(unsigned)(vblocks < 4096 ? vblocks : 4096), 256, 0, st>>>(g, w);
  const uint64_t rblocks = nfiles ? nfiles : 1;
  repair_kernel<<<(unsigned)(rblocks < 65535 ? rblocks : 65535), threads, smem, st>>>(g, dp, w);
  count_tiles_kernel<<<(unsigned)l.nitiles, kItemTile, 0, st>>>(w);
  emit_kernel<<<(unsigned)l.nitiles, kItemTile, 0, st>>>(g, w, d_cuts, cap,
                                                          d_cut_offsets, d_count);
  return cudaGetLastError() == cudaSuccess ? SEQCDC_OK : SEQCDC_ECUDA;
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

size_t seqcdc_workspace_size(const seqcdc_params_t *p, uint64_t total_bytes,
                             uint64_t nfiles, const seqcdc_tuning_t *tuning) {
  if (!params_ok(p)) return 0;
  return make_layout(p, total_bytes, nfiles, pick_segment(p, tuning)).total;
}

int seqcdc_chunk(const seqcdc_params_t *p, const uint8_t *d_in, uint64_t n,
                 uint64_t *d_cuts, uint64_t cap, uint64_t *d_count,
                 void *d_ws, size_t ws_bytes, const seqcdc_tuning_t *tuning,
                 void *stream) {
  if (!d_count) return SEQCDC_EINVAL;
  return run(p, d_in, n, nullptr, 1, d_cuts, cap, nullptr, d_count, d_ws,
             ws_bytes, tuning, stream);
}

int seqcdc_chunk_batch(const seqcdc_params_t *p, const uint8_t *d_data,
                       uint64_t total_bytes, const uint64_t *d_offsets,
                       uint64_t nfiles, uint64_t *d_cuts, uint64_t cap,
                       uint64_t *d_cut_offsets, void *d_ws, size_t ws_bytes,
                       const seqcdc_tuning_t *tuning, void *stream) {
  if (!d_offsets || !d_cut_offsets) return SEQCDC_EINVAL;
  return run(p, d_data, total_bytes, d_offsets, nfiles, d_cuts, cap,
             d_cut_offsets, nullptr, d_ws, ws_bytes, tuning, stream);
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
