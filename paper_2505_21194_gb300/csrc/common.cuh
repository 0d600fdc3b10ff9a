// common.cuh -- device helpers shared by the two chunking paths (the
// segment-map path in seqcdc.cu and the chain-walking path in walk.cu).
//
// The byte-pair classification of Sec. III.D: T[j] marks a target-order pair
// (b[j-1], b[j]) (strictly increasing in Increasing mode, strictly decreasing
// in Decreasing mode, bytes unsigned), O[j] the opposing order, and
// E[j] = T[j] & T[j-1] & ... & T[j-SeqLength+2] the last byte of a run of
// SeqLength bytes in target order.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace {

// Chunking parameters as the kernels take them (validated on the host:
// SeqLength 2..16, min_size >= 1, max_size <= 128 KiB).
struct DevParams {
  uint32_t mode;
  uint32_t R;   // seq_length
  uint32_t T;   // skip_trigger (0 = never)
  uint32_t S;   // skip_size
  uint32_t mn;  // min_size
  uint32_t mx;  // max_size
};

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

// Position (0..31) of the k-th set bit (1 <= k <= popc(x)); a branch-free
// binary descent over halves, quarters, ... of the word.
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t x, uint32_t k) {
  uint32_t pos = 0, c, t;
  c = __popc(x & 0xffffu); t = k > c; k -= t ? c : 0u; x >>= t ? 16 : 0; pos += t ? 16 : 0;
  c = __popc(x & 0xffu);   t = k > c; k -= t ? c : 0u; x >>= t ? 8 : 0;  pos += t ? 8 : 0;
  c = __popc(x & 0xfu);    t = k > c; k -= t ? c : 0u; x >>= t ? 4 : 0;  pos += t ? 4 : 0;
  c = __popc(x & 0x3u);    t = k > c; k -= t ? c : 0u; x >>= t ? 2 : 0;  pos += t ? 2 : 0;
  c = x & 1u;              t = k > c;                                    pos += t ? 1 : 0;
  return pos;
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

// Per-byte unsigned compares of a 4-byte word x with y, the same word shifted
// by one byte (y's byte k is the byte before x's byte k), answers in bit 7 of
// each byte.  Both come from one borrow-free subtraction: with
// z1 = (x | 0x80) - (y & 0x7f) - 1 per byte (0..0xfe), bit 7 of z1 is
// [x_low7 > y_low7] and z2 = 0xfe - z1 = (y | 0x80) - (x & 0x7f) - 1 gives
// [y_low7 > x_low7]; where the top bits differ they decide.
__device__ __forceinline__ void cmp_word(uint32_t x, uint32_t y, uint32_t &gt,
                                         uint32_t &lt) {
  const uint32_t z1 = (x | 0x80808080u) - (y & 0x7f7f7f7fu) - 0x01010101u;
  const uint32_t z2 = 0xfefefefeu - z1;
  gt = ((x & ~y) | (~(x ^ y) & z1)) & 0x80808080u;   // x > y per byte
  lt = ((y & ~x) | (~(x ^ y) & z2)) & 0x80808080u;   // x < y per byte
}

// Bit 7 of the 8 bytes of two words (a = bytes 0..3, b = bytes 4..7) -> bits
// 0..7 in byte order.  With a's bits moved to 3, 11, 19, 27 and b's at 7, 15,
// 23, 31, one multiplication by 1 + 2^7 + 2^14 + 2^21 lands them at 24..31 in
// order; the other partial products stay below bit 24 without overlapping.
__device__ __forceinline__ uint32_t gather8(uint32_t a, uint32_t b) {
  return (((a >> 4) | b) * 0x00204081u) >> 24;
}

// 32 bytes (two 16-byte vectors) with the byte before them -> T and O bits
// of the 32 positions (bit t = pair (byte t-1, byte t)).
__device__ __forceinline__ void classify32(uint4 v0, uint4 v1, uint32_t prev_byte,
                                           uint32_t mode, uint32_t &T,
                                           uint32_t &Ow) {
  uint32_t g0, l0, g1, l1, g2, l2, g3, l3, g4, l4, g5, l5, g6, l6, g7, l7;
  cmp_word(v0.x, (v0.x << 8) | (prev_byte & 0xffu), g0, l0);
  cmp_word(v0.y, __funnelshift_l(v0.x, v0.y, 8), g1, l1);
  cmp_word(v0.z, __funnelshift_l(v0.y, v0.z, 8), g2, l2);
  cmp_word(v0.w, __funnelshift_l(v0.z, v0.w, 8), g3, l3);
  cmp_word(v1.x, __funnelshift_l(v0.w, v1.x, 8), g4, l4);
  cmp_word(v1.y, __funnelshift_l(v1.x, v1.y, 8), g5, l5);
  cmp_word(v1.z, __funnelshift_l(v1.y, v1.z, 8), g6, l6);
  cmp_word(v1.w, __funnelshift_l(v1.z, v1.w, 8), g7, l7);
  const uint32_t up = gather8(g0, g1) | (gather8(g2, g3) << 8) |
                      (gather8(g4, g5) << 16) | (gather8(g6, g7) << 24);
  const uint32_t dn = gather8(l0, l1) | (gather8(l2, l3) << 8) |
                      (gather8(l4, l5) << 16) | (gather8(l6, l7) << 24);
  T = mode == 0 ? up : dn;
  Ow = mode == 0 ? dn : up;
}

// 16 bytes with the byte before them -> T and O bits of the 16 positions
// (bits 0..15; bit t = pair (byte t-1, byte t)).
__device__ __forceinline__ void classify16(uint4 v, uint32_t prev_byte, uint32_t mode,
                                           uint32_t &T, uint32_t &Ow) {
  uint32_t g0, l0, g1, l1, g2, l2, g3, l3;
  cmp_word(v.x, (v.x << 8) | (prev_byte & 0xffu), g0, l0);
  cmp_word(v.y, __funnelshift_l(v.x, v.y, 8), g1, l1);
  cmp_word(v.z, __funnelshift_l(v.y, v.z, 8), g2, l2);
  cmp_word(v.w, __funnelshift_l(v.z, v.w, 8), g3, l3);
  const uint32_t up = gather8(g0, g1) | (gather8(g2, g3) << 8);
  const uint32_t dn = gather8(l0, l1) | (gather8(l2, l3) << 8);
  T = mode == 0 ? up : dn;
  Ow = mode == 0 ? dn : up;
}

// E at position t needs T at t, t-1, ..., t-(R-2); `pt` holds the T bits of
// the 32 positions before.
__device__ __forceinline__ uint32_t run_ends(uint32_t pt, uint32_t T, uint32_t R) {
  if (R == 5)  // the paper's SeqLength at every setting (Table I)
    return T & __funnelshift_l(pt, T, 1) & __funnelshift_l(pt, T, 2) &
           __funnelshift_l(pt, T, 3);
  uint32_t ew = T;
  for (uint32_t k = 1; k + 1 < R; ++k) ew &= __funnelshift_l(pt, T, k);
  return ew;
}

// Record a measurement event on `st`.  While the stream is being captured
// into a CUDA graph the record becomes an event node that fires on every
// launch of the graph (an external record), so that the events bracket the
// kernel in each replay.
inline void record_event(cudaEvent_t ev, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
  else
    cudaEventRecord(ev, st);
}

}  // namespace
