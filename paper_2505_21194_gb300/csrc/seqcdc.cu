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

#include "seqcdc.h"

namespace {

// ---------------------------------------------------------------------------
// Limits and layout constants.
// ---------------------------------------------------------------------------
constexpr int kMaxEntries = 512;   // natural entries walked per item
constexpr int kMaxNodes = 1024;    // distinct cut positions per item walk
constexpr int kHashSlots = 2048;   // open-addressing slots (power of two)
constexpr int kMaxImage = 32;      // distinct exits published per item (one per lane)
constexpr int kFileTile = 1024;    // files per plan block
constexpr int kItemTile = 256;     // items per compaction block
constexpr uint32_t kMaxSeqLength = 16;
constexpr uint64_t kMaxMaxSize = 262144;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on any device wait

// Item state bits (set once, in this order of availability).
constexpr uint32_t F_IMG = 1u;     // image (distinct exits) published
constexpr uint32_t F_NOIMG = 2u;   // no image (more than kMaxImage exits)
constexpr uint32_t F_AGG = 4u;     // map predecessor image -> exits published
constexpr uint32_t F_NOAGG = 8u;   // no such map (predecessor had no image)
constexpr uint32_t F_INCL = 16u;   // true exit, entry and cuts published

constexpr uint16_t kNil = 0xFFFFu;
constexpr uint32_t kNone = 0xFFFFFFFFu;

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
  uint32_t stats[8];  // see seqcdc_stats()
  uint32_t pad[53];
};

enum : uint32_t {
  ST_ITEMS = 0,         // items processed
  ST_ABNORMAL = 1,      // items whose natural entries could not all be walked
  ST_NOIMG = 2,         // items with more distinct exits than published
  ST_LB_WAITS = 3,      // look-backs that had to wait for a true exit
  ST_INCONSISTENT = 4,  // items whose entry disagreed with the predecessor
  ST_RECOMPUTED = 5,    // items re-chunked by the repair pass
  ST_REPLAYED = 6,      // emissions by stepping (entry was not a natural cut)
  ST_LB_STEPS = 7,      // total look-back depth
};

struct Layout {
  size_t hdr, seg_base, ftile, state, incl, entry, first_bad, count, img_n,
      img, agg, slot, itile, total;
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
  uint32_t v = ld_acquire(flag);
  if (v & mask) return v;
  const uint64_t t0 = global_ns();
  uint32_t backoff = 32;
  for (uint64_t it = 0; it < (1ull << 32); ++it) {
    __nanosleep(backoff);
    if (backoff < 512) backoff <<= 1;
    v = ld_acquire(flag);
    if (v & mask) return v;
    if (global_ns() - t0 > kWaitNs) break;
  }
  atomicExch(&hdr->status, (uint32_t)SEQCDC_ETIMEOUT);
  return 0;
}

// Per-byte "a > b" for four unsigned bytes; the answer is in bit 7 of each
// byte, the other bits are garbage.  Low seven bits are compared with a
// borrow-free subtraction ((a | 0x80) - (b & 0x7f) - 1 stays within 0..0xff),
// the high bits decide when they differ.
__device__ __forceinline__ uint32_t gt_hi(uint32_t a, uint32_t b) {
  const uint32_t z = (a | 0x80808080u) - (b & 0x7f7f7f7fu) - 0x01010101u;
  return (a & ~b) | (~(a ^ b) & z);
}

// Gather bit 7 of each byte into bits 0..3 (byte k -> bit k).
__device__ __forceinline__ uint32_t pack4(uint32_t m) {
  return ((m & 0x80808080u) * 0x00204081u) >> 28;
}

// Position (0..31) of the k-th set bit (1 <= k <= popc(x)).
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

// Target / opposing masks (16 positions) for the 16 bytes in v, given the
// byte before them.  Bit t refers to the pair (byte t-1, byte t).
__device__ __forceinline__ void classify16(uint32_t prev_byte, uint4 v,
                                           uint32_t mode, uint32_t &T16,
                                           uint32_t &O16) {
  const uint32_t x0 = v.x, x1 = v.y, x2 = v.z, x3 = v.w;
  const uint32_t y0 = (x0 << 8) | (prev_byte & 0xffu);
  const uint32_t y1 = __funnelshift_l(x0, x1, 8);
  const uint32_t y2 = __funnelshift_l(x1, x2, 8);
  const uint32_t y3 = __funnelshift_l(x2, x3, 8);
  const uint32_t up = pack4(gt_hi(x0, y0)) | (pack4(gt_hi(x1, y1)) << 4) |
                      (pack4(gt_hi(x2, y2)) << 8) | (pack4(gt_hi(x3, y3)) << 12);
  const uint32_t dn = pack4(gt_hi(y0, x0)) | (pack4(gt_hi(y1, x1)) << 4) |
                      (pack4(gt_hi(y2, x2)) << 8) | (pack4(gt_hi(y3, x3)) << 12);
  T16 = mode == 0 ? up : dn;
  O16 = mode == 0 ? dn : up;
}

// 16 input bytes at global byte index gi (16-aligned); bytes outside
// [0, total) read as zero.
__device__ __forceinline__ uint4 load16(const uint8_t *data, int64_t gi,
                                        uint64_t total) {
  if (gi >= 0 && (uint64_t)gi + 16 <= total) {
    return __ldg(reinterpret_cast<const uint4 *>(data + gi));
  }
  uint32_t w[4] = {0, 0, 0, 0};
  for (int t = 0; t < 16; ++t) {
    const int64_t a = gi + t;
    if (a >= 0 && (uint64_t)a < total) w[t >> 2] |= (uint32_t)data[a] << (8 * (t & 3));
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Exclusive block scan of one value per thread (blockDim <= 1024).
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t *scratch,
                                    uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  uint32_t x = v;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t s = lane < nwarps ? scratch[lane] : 0u;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
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
// Bitmaps of one item in shared memory.  Positions are relative to the window
// base B (file-relative): rel = pos - B; word w covers rel 32w .. 32w+31; a
// block is 8 words (256 positions).
//   E, O    run-end and opposing-pair bits
//   eany    bit b set when block b has an E bit
//   ocnt    number of O bits in block b
// ---------------------------------------------------------------------------
struct Bits {
  const uint32_t *E;
  const uint32_t *O;
  const uint32_t *eany;
  const uint16_t *ocnt;
};

// First E position in [x, limit), or kNone.
__device__ __forceinline__ uint32_t first_E(const Bits &b, uint32_t x,
                                            uint32_t limit) {
  if (x >= limit) return kNone;
  const uint32_t wl = (limit - 1) >> 5;
  uint32_t w = x >> 5;
  uint32_t m = b.E[w] & (~0u << (x & 31));
  while (true) {
    if (m) {
      const uint32_t pos = (w << 5) + (__ffs(m) - 1);
      return pos < limit ? pos : kNone;
    }
    if (w >= wl) return kNone;
    ++w;
    if ((w & 7) == 0) {  // block boundary: jump to the next block with E bits
      const uint32_t bl = wl >> 3;
      uint32_t bi = w >> 3;
      uint32_t fw = bi >> 5;
      uint32_t fm = b.eany[fw] & (~0u << (bi & 31));
      while (!fm) {
        ++fw;
        if ((fw << 5) > bl) return kNone;
        fm = b.eany[fw];
      }
      bi = (fw << 5) + (__ffs(fm) - 1);
      if (bi > bl) return kNone;
      w = bi << 3;
    }
    m = b.E[w];
  }
}

// Position of the need-th O bit at or after x (need >= 1), if < limit; else kNone.
__device__ __forceinline__ uint32_t nth_O(const Bits &b, uint32_t x,
                                          uint32_t need, uint32_t limit) {
  if (x >= limit) return kNone;
  const uint32_t wl = (limit - 1) >> 5;
  uint32_t w = x >> 5;
  uint32_t m = b.O[w] & (~0u << (x & 31));
  uint32_t c = __popc(m);
  while (c < need) {
    need -= c;
    if (w >= wl) return kNone;
    ++w;
    if ((w & 7) == 0) {  // whole blocks that cannot hold the need-th bit
      while (w + 8 <= wl + 1 && b.ocnt[w >> 3] < need) {
        need -= b.ocnt[w >> 3];
        w += 8;
      }
      if (w > wl) return kNone;
    }
    m = b.O[w];
    c = __popc(m);
  }
  const uint32_t pos = (w << 5) + nth_set_bit(m, need);
  return pos < limit ? pos : kNone;
}

// One chunk: from chunk start c (rel) return its end (rel).  `end_rel` is the
// rel position of the file end.
__device__ uint32_t chunk_step(const Bits &b, const DevParams &p, uint32_t c,
                               uint32_t end_rel) {
  const uint32_t limit = (end_rel - c > p.mx) ? c + p.mx : end_rel;
  uint32_t i = c + (p.mn > p.R ? p.mn - p.R : 0u);
  while (i + 1 < limit) {
    const uint32_t s = p.T ? nth_O(b, i + 1, p.T, limit) : kNone;
    const uint32_t e = first_E(b, i + p.R - 1, s == kNone ? limit : s);
    if (e != kNone) return e + 1;     // boundary run ends first (Sec. III.A)
    if (s == kNone) break;
    i = s + 1 + p.S;                  // content-defined skip (Sec. III.C)
  }
  return limit;                       // max size or end of input (Sec. IV)
}

__device__ __forceinline__ uint32_t hash_pos(uint32_t x) {
  return (x * 2654435761u) >> (32 - 11);  // kHashSlots = 2048
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
struct SegShared {
  uint32_t item, file, seg, nitems, first_item;
  int64_t B;          // window base (file-relative); global index of rel 0 is 16-aligned
  uint64_t p_s, q_s, n_f, gbase;
  uint32_t W, NB;     // bitmap words, blocks
  uint32_t K;         // natural entries
  uint32_t nnodes, nact, nnew, abnormal, nimg, npred, pred_flags;
  uint32_t scratch[32];
  uint64_t true_entry;
};

struct SegSmem {
  uint32_t *E, *O, *eany;
  uint16_t *ocnt;
  uint32_t *node_pos;     // kMaxNodes
  uint16_t *node_next;    // kMaxNodes
  uint16_t *hslot;        // kHashSlots (reused as jmp after the walk)
  uint16_t *act, *act2;   // kMaxNodes each
  uint64_t *img_local;    // kMaxImage
  uint64_t *agg_local;    // kMaxImage
};

__host__ __device__ inline uint32_t nblocks(uint32_t W) { return (W + 7) / 8; }

__device__ __forceinline__ SegSmem carve(unsigned char *raw, uint32_t W) {
  SegSmem m;
  const uint32_t NB = nblocks(W);
  m.E = reinterpret_cast<uint32_t *>(raw);
  m.O = m.E + W;
  m.eany = m.O + W;
  m.node_pos = m.eany + (NB + 31) / 32;
  m.img_local = reinterpret_cast<uint64_t *>(
      reinterpret_cast<uintptr_t>(m.node_pos + kMaxNodes + 1) & ~(uintptr_t)7);
  m.agg_local = m.img_local + kMaxImage;
  m.node_next = reinterpret_cast<uint16_t *>(m.agg_local + kMaxImage);
  m.hslot = m.node_next + kMaxNodes;
  m.act = m.hslot + kHashSlots;
  m.act2 = m.act + kMaxNodes;
  m.ocnt = m.act2 + kMaxNodes;
  return m;
}

__host__ __device__ inline size_t seg_smem_bytes_for(uint32_t W) {
  const uint32_t NB = nblocks(W);
  return (size_t)W * 8 + ((NB + 31) / 32) * 4 + (kMaxNodes + 1) * 4 + 8 +
         kMaxImage * 16 + kMaxNodes * 2 + kHashSlots * 2 + kMaxNodes * 4 +
         (size_t)NB * 2 + 16;
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
  sh.NB = nblocks(sh.W);
  sh.abnormal = 0;
  sh.nnodes = 0;
  sh.K = 0;
  sh.nimg = 0;
  sh.npred = 0;
}

__device__ __forceinline__ Bits bits_of(const SegSmem &m) {
  return Bits{m.E, m.O, m.eany, m.ocnt};
}

// E and O bitmaps of the window [B, B + 32 W) and their block summaries.
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
  __syncthreads();
  // Block summaries; each warp covers 32 consecutive blocks per pass.
  const uint32_t NB = sh.NB;
  for (uint32_t b0 = warp * 32; b0 < NB; b0 += nwarps * 32) {
    const uint32_t b = b0 + lane;
    uint32_t any = 0, cnt = 0;
    if (b < NB) {
      const uint32_t w0 = b * 8, w1 = min(w0 + 8, W);
      for (uint32_t w = w0; w < w1; ++w) {
        any |= m.E[w];
        cnt += __popc(m.O[w]);
      }
      m.ocnt[b] = (uint16_t)cnt;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, any != 0);
    if (lane == 0) m.eany[b0 >> 5] = bal;
  }
}

// Entry candidates, then the walk of every entry's chain to its exit with
// merging, then each entry's exit by pointer jumping (left in hslot[0..n) as
// the terminal node index).  All threads.  Sets sh.abnormal when the entries
// or nodes do not fit.
__device__ void seg_walk(SegShared &sh, const DevParams &p, const SegSmem &m) {
  const int tid = threadIdx.x, nthreads = blockDim.x;
  const int64_t B = sh.B;
  const uint64_t n_f = sh.n_f, p_s = sh.p_s;
  const uint32_t end_rel = (uint32_t)((int64_t)n_f - B);
  const uint32_t q_rel = (uint32_t)((int64_t)sh.q_s - B);
  const uint32_t ps_rel = (uint32_t)((int64_t)p_s - B);
  const Bits bits = bits_of(m);

  // Item 0 of a file starts at the file start; any other item may be entered
  // at every natural cut x = e + 1 (E[e] set) with p_s <= x < p_s + max_size.
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
  if (sh.abnormal) return;

  const uint32_t K = sh.K;
  for (int i = tid; i < kHashSlots; i += nthreads) m.hslot[i] = kNil;
  for (int i = tid; i < kMaxNodes; i += nthreads) m.node_next[i] = kNil;
  if (tid == 0) {
    sh.nnodes = K;
    sh.nact = 0;
    sh.nnew = 0;
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
          m.node_pos[nid] = kNone;  // lost the slot; the winner may match
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
    }
    uint16_t *tmp = cur_act;
    cur_act = nxt_act;
    nxt_act = tmp;
    __syncthreads();
  }
  if (sh.abnormal) return;

  // Terminal nodes are the exits; pointer jumping gives every node its
  // terminal.  A path can pass through several merged chains, so its length
  // is bounded by the node count, not by the number of rounds.
  const uint32_t nn = min(sh.nnodes, (uint32_t)kMaxNodes);
  uint16_t *jmp = m.hslot;
  for (uint32_t n = tid; n < nn; n += nthreads) {
    const uint16_t nx = m.node_next[n];
    jmp[n] = (nx == kNil) ? (uint16_t)n : nx;
    if (nx == kNil && m.node_pos[n] != kNone) {
      const uint32_t idx = atomicAdd(&sh.nimg, 1u);
      if (idx < (uint32_t)kMaxImage) m.img_local[idx] = (uint64_t)(B + (int64_t)m.node_pos[n]);
    }
  }
  __syncthreads();
  for (uint32_t r = 1; r < 2 * nn; r <<= 1) {
    for (uint32_t n = tid; n < nn; n += nthreads) m.act[n] = jmp[jmp[n]];
    __syncthreads();
    for (uint32_t n = tid; n < nn; n += nthreads) jmp[n] = m.act[n];
    __syncthreads();
  }
}

// Exit of this item from entry x (file-relative): follow the walked nodes when
// x is a natural entry, else step the chunker on the bitmaps.  One thread.
__device__ uint64_t seg_exit_from(const SegShared &sh, const DevParams &p,
                                  const SegSmem &m, uint64_t x) {
  const int64_t B = sh.B;
  const uint32_t xr = (uint32_t)((int64_t)x - B);
  if (!sh.abnormal) {
    uint32_t lo = 0, hi = sh.K;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      const uint32_t v = m.node_pos[mid];
      if (v == xr) return (uint64_t)(B + (int64_t)m.node_pos[m.hslot[mid]]);
      if (v < xr) lo = mid + 1; else hi = mid;
    }
  }
  const Bits bits = bits_of(m);
  const uint32_t end_rel = (uint32_t)((int64_t)sh.n_f - B);
  const uint32_t q_rel = (uint32_t)((int64_t)sh.q_s - B);
  uint32_t c = xr;
  while (c < q_rel) c = chunk_step(bits, p, c, end_rel);
  return (uint64_t)(B + (int64_t)c);
}

// Publish the image: distinct exits over the walked entries.  All threads.
__device__ void seg_publish_image(SegShared &sh, const SegSmem &m,
                                  const WsPtrs &ws) {
  const int tid = threadIdx.x;
  const uint32_t item = sh.item;
  const uint32_t nimg = sh.nimg;
  const bool too_many = nimg > (uint32_t)kMaxImage;
  if (!too_many)
    for (uint32_t k = tid; k < nimg; k += blockDim.x)
      ws.img[(uint64_t)item * kMaxImage + k] = m.img_local[k];
  __syncthreads();
  if (tid == 0) {
    ws.img_n[item] = too_many ? 0u : nimg;
    __threadfence();
    atomicOr(&ws.state[item], too_many ? F_NOIMG : F_IMG);
    if (too_many) atomicAdd(&ws.hdr->stats[ST_NOIMG], 1u);
  }
}

// Map from the predecessor's image to this item's exits (the "aggregate" of
// the decoupled look-back).  For an item whose natural entries could not be
// walked, the map's values also become its image.  All threads.
__device__ void seg_publish_agg(SegShared &sh, const DevParams &p,
                                const SegSmem &m, const WsPtrs &ws) {
  const int tid = threadIdx.x;
  const uint32_t item = sh.item;
  if (tid == 0) {
    const uint32_t st = wait_any(&ws.state[item - 1], F_IMG | F_NOIMG, ws.hdr);
    sh.pred_flags = st;
    sh.npred = (st & F_IMG) ? __ldcg(&ws.img_n[item - 1]) : 0u;
  }
  __syncthreads();
  const uint32_t npred = sh.npred;
  const bool ok = (sh.pred_flags & F_IMG) != 0;
  if (ok) {
    ld_acquire(&ws.state[item - 1]);
    for (uint32_t j = tid; j < npred; j += blockDim.x) {
      const uint64_t y = __ldcg(&ws.img[(uint64_t)(item - 1) * kMaxImage + j]);
      const uint64_t ex = seg_exit_from(sh, p, m, y);
      m.agg_local[j] = ex;
      ws.agg[(uint64_t)item * kMaxImage + j] = ex;
    }
  }
  __syncthreads();
  if (tid == 0) {
    if (sh.abnormal) {
      // Image of an item without a full walk: the distinct mapped exits.
      uint32_t n = 0;
      if (ok) {
        for (uint32_t j = 0; j < npred; ++j) {
          bool seen = false;
          for (uint32_t k = 0; k < n; ++k) seen |= (m.img_local[k] == m.agg_local[j]);
          if (!seen) m.img_local[n++] = m.agg_local[j];
        }
        for (uint32_t k = 0; k < n; ++k) ws.img[(uint64_t)item * kMaxImage + k] = m.img_local[k];
      }
      ws.img_n[item] = n;
      __threadfence();
      atomicOr(&ws.state[item], ok ? (F_IMG | F_AGG) : (F_NOIMG | F_NOAGG));
      if (!ok) atomicAdd(&ws.hdr->stats[ST_NOIMG], 1u);
    } else {
      __threadfence();
      atomicOr(&ws.state[item], ok ? F_AGG : F_NOAGG);
    }
  }
}

// True entry by decoupled look-back (warp 0).  Going back from item-1, each
// predecessor k either has published its true exit (stop), or its map from
// the image of k-1 to its exits (compose and continue), or no map (wait for
// its true exit).  The composite is held as one value per lane: lane j holds
// the exit of item-1 reached from value j of the current image.
__device__ uint64_t seg_lookback(SegShared &sh, const WsPtrs &ws) {
  const int lane = threadIdx.x & 31;
  const uint32_t item = sh.item;
  uint32_t k = item - 1;
  uint64_t comp = 0;        // per lane: composite value (valid if have)
  bool have = false;        // composite defined for this lane
  bool started = false;     // at least one map composed
  uint32_t steps = 0;
  uint64_t x = 0;
  bool waited = false;
  while (true) {
    // Lane 0 waits; every lane then acquires the flag for its own reads, but
    // all lanes branch on lane 0's snapshot (flags only gain bits, and lanes
    // acting on different snapshots would diverge around warp shuffles).
    uint32_t st = 0;
    if (lane == 0) st = wait_any(&ws.state[k], F_INCL | F_AGG | F_NOAGG, ws.hdr);
    st = __shfl_sync(0xffffffffu, st, 0);
    if (st == 0) { x = sh.p_s; break; }  // timed out; status is recorded
    (void)ld_acquire(&ws.state[k]);
    __syncwarp();
    if (!(st & F_INCL) && (st & F_NOAGG)) {
      if (lane == 0) st = wait_any(&ws.state[k], F_INCL, ws.hdr);
      st = __shfl_sync(0xffffffffu, st, 0);
      waited = true;
      if (st == 0) { x = sh.p_s; break; }
      (void)ld_acquire(&ws.state[k]);
      __syncwarp();
    }
    if (st & F_INCL) {
      const uint64_t e = __ldcg(&ws.incl[k]);  // true exit of k = entry of k+1
      if (!started) { x = e; break; }
      // Find e in the image of k (the domain of the composite).
      const uint32_t n = __ldcg(&ws.img_n[k]);
      const uint64_t v = (lane < (int)n) ? __ldcg(&ws.img[(uint64_t)k * kMaxImage + lane]) : ~0ull;
      const uint32_t hit = __ballot_sync(0xffffffffu, lane < (int)n && v == e && have);
      if (hit) {
        x = __shfl_sync(0xffffffffu, comp, __ffs(hit) - 1);
        break;
      }
      // The true exit of k is outside the composite's domain: wait for the
      // true exit of item-1 instead.
      if (lane == 0) st = wait_any(&ws.state[item - 1], F_INCL, ws.hdr);
      st = __shfl_sync(0xffffffffu, st, 0);
      waited = true;
      if (st) {
        (void)ld_acquire(&ws.state[item - 1]);
        __syncwarp();
        x = __ldcg(&ws.incl[item - 1]);
      } else {
        x = sh.p_s;
      }
      break;
    }
    // F_AGG: map from the image of k-1 to the exits of k.
    const uint32_t n_agg = __ldcg(&ws.img_n[k - 1]);
    const uint64_t a = (lane < (int)n_agg) ? __ldcg(&ws.agg[(uint64_t)k * kMaxImage + lane]) : 0;
    if (!started) {
      comp = a;
      have = lane < (int)n_agg;
      started = true;
    } else {
      // New composite over image(k-1): lane j -> comp at the index of a_j in image(k).
      const uint32_t n_img = __ldcg(&ws.img_n[k]);
      const uint64_t im = (lane < (int)n_img) ? __ldcg(&ws.img[(uint64_t)k * kMaxImage + lane]) : ~0ull;
      uint64_t nc = 0;
      bool nh = false;
      for (uint32_t j = 0; j < n_img; ++j) {
        const uint64_t imj = __shfl_sync(0xffffffffu, im, j);
        const uint64_t cj = __shfl_sync(0xffffffffu, comp, j);
        const bool hj = __shfl_sync(0xffffffffu, have, j);
        if (!nh && lane < (int)n_agg && a == imj && hj) { nc = cj; nh = true; }
      }
      comp = nc;
      have = nh;
    }
    ++steps;
    // A constant composite settles the entry whichever image value was true
    // (under the same tabulated-entry assumption the verify pass checks).
    {
      const uint32_t hv = __ballot_sync(0xffffffffu, have);
      if (hv == 0) {  // nothing composes any more: wait for item-1's true exit
        if (lane == 0) st = wait_any(&ws.state[item - 1], F_INCL, ws.hdr);
        st = __shfl_sync(0xffffffffu, st, 0);
        waited = true;
        if (st) {
          (void)ld_acquire(&ws.state[item - 1]);
          __syncwarp();
          x = __ldcg(&ws.incl[item - 1]);
        } else {
          x = sh.p_s;
        }
        break;
      }
      const uint64_t c0 = __shfl_sync(0xffffffffu, comp, __ffs(hv) - 1);
      if (__all_sync(0xffffffffu, !have || comp == c0)) {
        x = c0;
        break;
      }
    }
    --k;  // k > first item: the first item publishes F_INCL, never F_AGG
  }
  if (lane == 0) {
    atomicAdd(&ws.hdr->stats[ST_LB_STEPS], steps);
    if (waited) atomicAdd(&ws.hdr->stats[ST_LB_WAITS], 1u);
  }
  return x;
}

// Emission from entry x: the cuts in (x, exit] into the item's slot, then the
// entry, exit and count, then F_INCL.  Thread 0.
__device__ void seg_emit(SegShared &sh, const DevParams &p, const SegSmem &m,
                         const WsPtrs &ws, uint64_t x, bool use_nodes) {
  const int64_t B = sh.B;
  const Bits bits = bits_of(m);
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
    atomicAdd(&ws.hdr->stats[ST_REPLAYED], 1u);
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
  atomicOr(&ws.state[item], F_INCL);
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
    atomicAdd(&ws.hdr->stats[ST_ITEMS], 1u);
  }
  __syncthreads();
  const SegSmem m = carve(smem_raw, sh.W);
  seg_bitmaps(sh, g, p, m);
  __syncthreads();
  seg_walk(sh, p, m);
  __syncthreads();
  if (sh.abnormal) {
    if (tid == 0) atomicAdd(&ws.hdr->stats[ST_ABNORMAL], 1u);
  } else {
    seg_publish_image(sh, m, ws);
  }
  __syncthreads();
  if (sh.seg == 0) {
    if (tid == 0) {
      if (sh.abnormal) {
        // Image of an unwalked first item: its single exit from the file start.
        const uint64_t ex = seg_exit_from(sh, p, m, 0);
        ws.img[(uint64_t)sh.item * kMaxImage] = ex;
        ws.img_n[sh.item] = 1;
        __threadfence();
        atomicOr(&ws.state[sh.item], F_IMG);
      }
      sh.true_entry = 0;
    }
  } else {
    seg_publish_agg(sh, p, m, ws);
    __syncthreads();
    if (tid < 32) {
      const uint64_t x = seg_lookback(sh, ws);
      if (tid == 0) sh.true_entry = x;
    }
  }
  __syncthreads();
  if (tid == 0) seg_emit(sh, p, m, ws, sh.true_entry, !sh.abnormal);
}

// Verify: item s of a file is consistent when its entry equals the exit its
// predecessor computed.  By induction from the file start (always a true
// entry), a file whose items are all consistent is exact.  The first
// inconsistent item of each file is recorded for the repair pass.
__global__ void verify_kernel(Geom g, WsPtrs ws) {
  const uint32_t nitems = ws.hdr->nitems;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nitems;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t f = find_file(ws.seg_base, g.nfiles, (uint32_t)i);
    const uint32_t s = (uint32_t)i - ws.seg_base[f];
    bool ok = (ws.state[i] & F_INCL) != 0;
    if (ok && s > 0) ok = ws.entry[i] == ws.incl[i - 1];
    if (ok && s == 0) ok = ws.entry[i] == 0;
    if (!ok) {
      atomicMin(&ws.first_bad[f], s);
      atomicAdd(&ws.hdr->stats[ST_INCONSISTENT], 1u);
    }
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
    uint64_t cur = fb ? ws.incl[base + fb - 1] : 0;
    for (uint32_t s = fb; s < nseg; ++s) {
      const uint32_t item = base + s;
      if (tid == 0) {
        s_run = !((ws.state[item] & F_INCL) && ws.entry[item] == cur);
        if (s_run) {
          seg_setup(sh, g, p, item, (uint32_t)f, s, base);
          sh.abnormal = 1;  // no walk: emit by stepping
          atomicAdd(&ws.hdr->stats[ST_RECOMPUTED], 1u);
        }
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
  __shared__ uint64_t red64[32];
  __shared__ uint64_t s_prefix;
  __shared__ uint32_t offs[kItemTile + 1];
  const uint32_t nitems = ws.hdr->nitems;
  const uint64_t lo = (uint64_t)blockIdx.x * kItemTile;
  uint64_t part = 0;
  for (uint64_t t = threadIdx.x; t < blockIdx.x; t += blockDim.x) part += ws.itile[t];
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
  for (int it = warp; it < kItemTile; it += blockDim.x >> 5) {
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
  // CSR offsets of the files whose first item index falls in [lo, lo+tile).
  const uint64_t hi = lo + kItemTile;
  if (lo <= nitems) {
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

uint32_t pick_segment(const seqcdc_tuning_t *t) {
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

uint32_t max_words(uint32_t L, uint64_t mx) {
  return (uint32_t)((L + mx + 64 + 31) / 32 + 2);
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
  w.agg = reinterpret_cast<uint64_t *>(b + l.agg);
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
  const uint32_t L = pick_segment(tuning);
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
  const size_t smem = seg_smem_bytes_for(max_words(L, p->max_size));
  if (smem > 227 * 1024) return SEQCDC_ERANGE;
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
  plan_tiles_kernel<<<(unsigned)l.nftiles, 256, 0, st>>>(g, w);
  plan_scan_kernel<<<(unsigned)l.nftiles, 256, 0, st>>>(g, w, l.nftiles, l.imax);
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
  return make_layout(p, total_bytes, nfiles, pick_segment(tuning)).total;
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
