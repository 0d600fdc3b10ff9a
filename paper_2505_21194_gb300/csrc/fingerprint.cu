/*
 * fingerprint.cu -- SHA-256 fingerprints of chunks and a device hash table
 * that counts the distinct ones: the deduplication step that follows
 * content-defined chunking (Sec. II: chunks are fingerprinted and a chunk
 * whose fingerprint is already stored is not stored again).
 *
 * SHA-256 is written from its definition (FIPS 180-4: padding Sec. 5.1.1,
 * message schedule and compression Sec. 6.2.2, functions Sec. 4.1.2).  Its
 * constants (Sec. 4.2.2, Sec. 5.3.3) are derived here from the first primes
 * with exact integer roots instead of being listed.
 *
 * A thread hashes whole chunks (the 64-byte blocks of a chunk are sequential
 * by definition, and a batch holds far more chunks than the GPU has lanes),
 * several in a row, one block per iteration, so the lanes of a warp stay busy
 * whatever the chunk sizes.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "seqcdc.h"

namespace {

__constant__ uint32_t c_K[64];
__constant__ uint32_t c_H0[8];

constexpr uint32_t kEmpty = 0xffffffffu;
constexpr int kMaxDevices = 64;

// floor(x^(1/k)) for k = 2 or 3 and x < 2^110, by bisection.
unsigned __int128 iroot(unsigned __int128 x, int k) {
  unsigned __int128 lo = 0, hi = (unsigned __int128)1 << (k == 2 ? 56 : 38);
  while (hi - lo > 1) {
    const unsigned __int128 mid = (lo + hi) >> 1;
    const unsigned __int128 pw = (k == 2) ? mid * mid : mid * mid * mid;
    if (pw <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// First 32 bits of the fractional parts of the cube roots of the first 64
// primes (K) and of the square roots of the first 8 primes (H0):
// floor(r * 2^32) = floor((p * 2^(32 k))^(1/k)), whose low 32 bits are the
// fraction's.
void sha256_constants(uint32_t K[64], uint32_t H0[8]) {
  uint32_t primes[64];
  int n = 0;
  for (uint32_t c = 2; n < 64; ++c) {
    bool prime = true;
    for (uint32_t d = 2; d * d <= c; ++d)
      if (c % d == 0) { prime = false; break; }
    if (prime) primes[n++] = c;
  }
  for (int i = 0; i < 64; ++i)
    K[i] = (uint32_t)(iroot((unsigned __int128)primes[i] << 96, 3) & 0xffffffffu);
  for (int i = 0; i < 8; ++i)
    H0[i] = (uint32_t)(iroot((unsigned __int128)primes[i] << 64, 2) & 0xffffffffu);
}

// Upload the constants once per device.
bool constants_ready() {
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return true;
  uint32_t K[64], H0[8];
  sha256_constants(K, H0);
  if (cudaMemcpyToSymbol(c_K, K, sizeof(K)) != cudaSuccess ||
      cudaMemcpyToSymbol(c_H0, H0, sizeof(H0)) != cudaSuccess)
    return false;
  done[dev] = true;
  return true;
}

__device__ __forceinline__ uint32_t rotr(uint32_t x, int n) { return __funnelshift_r(x, x, n); }
__device__ __forceinline__ uint32_t bswap(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// One application of the compression function to state h and block w
// (16 big-endian words).
__device__ __forceinline__ void compress(uint32_t h[8], uint32_t w[16]) {
  uint32_t a = h[0], b = h[1], c = h[2], d = h[3];
  uint32_t e = h[4], f = h[5], g = h[6], k = h[7];
#pragma unroll
  for (int t = 0; t < 64; ++t) {
    if (t >= 16) {
      const uint32_t w2 = w[(t - 2) & 15], w15 = w[(t - 15) & 15];
      const uint32_t s1 = rotr(w2, 17) ^ rotr(w2, 19) ^ (w2 >> 10);
      const uint32_t s0 = rotr(w15, 7) ^ rotr(w15, 18) ^ (w15 >> 3);
      w[t & 15] += s1 + w[(t - 7) & 15] + s0;
    }
    const uint32_t S1 = rotr(e, 6) ^ rotr(e, 11) ^ rotr(e, 25);
    const uint32_t ch = (e & f) ^ (~e & g);
    const uint32_t t1 = k + S1 + ch + c_K[t] + w[t & 15];
    const uint32_t S0 = rotr(a, 2) ^ rotr(a, 13) ^ rotr(a, 22);
    const uint32_t mj = (a & b) ^ (a & c) ^ (b & c);
    const uint32_t t2 = S0 + mj;
    k = g; g = f; f = e; e = d + t1;
    d = c; c = b; b = a; a = t1 + t2;
  }
  h[0] += a; h[1] += b; h[2] += c; h[3] += d;
  h[4] += e; h[5] += f; h[6] += g; h[7] += k;
}

// Little-endian 32-bit word of data at byte q (4-aligned), bytes past
// `total` read as zero.
__device__ __forceinline__ uint32_t word_at(const uint8_t *data, uint64_t q, uint64_t total) {
  if (q + 4 <= total) return __ldg(reinterpret_cast<const uint32_t *>(data + q));
  uint32_t v = 0;
  for (int j = 0; j < 4; ++j)
    if (q + j < total) v |= (uint32_t)data[q + j] << (8 * j);
  return v;
}

// Absolute byte range [a, b) of chunk i of a CSR batch.
__device__ __forceinline__ void chunk_range(const uint64_t *offsets, uint64_t nfiles,
                                            const uint64_t *cuts, const uint64_t *cut_offsets,
                                            uint64_t i, uint64_t &a, uint64_t &b) {
  uint64_t lo = 0, hi = nfiles;  // file f: cut_offsets[f] <= i < cut_offsets[f + 1]
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (cut_offsets[mid] <= i) lo = mid; else hi = mid;
  }
  const uint64_t fbase = offsets[lo];
  a = fbase + (i > cut_offsets[lo] ? cuts[i - 1] : 0);
  b = fbase + cuts[i];
}

// Pass 1: the byte range [a, b) of every chunk, parked in the first 16 bytes
// of the chunk's digest slot (pass 2 reads it before it writes the digest).
__global__ void chunk_ranges_kernel(const uint64_t *offsets, uint64_t nfiles,
                                    const uint64_t *cuts, const uint64_t *cut_offsets,
                                    uint64_t ncuts, uint32_t *digests) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ncuts;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t a, b;
    chunk_range(offsets, nfiles, cuts, cut_offsets, i, a, b);
    reinterpret_cast<ulonglong2 *>(digests)[2 * i] = make_ulonglong2(a, b);
  }
}

// Block `off` (a multiple of 64) of the padded message of the chunk at
// [a, a + len): data bytes, the 0x80 marker, zeros, and in the last block the
// bit length (Sec. 5.1.1).  Whole data blocks come from 16 or 17 aligned
// words funnel-shifted to the chunk's byte offset.
__device__ __forceinline__ void message_block(const uint8_t *data, uint64_t total,
                                              uint64_t a, uint64_t len, uint64_t off,
                                              uint64_t padded, uint32_t w[16]) {
  if (off + 64 <= len) {
    const uint64_t q = a + off;
    const uint64_t q4 = q & ~3ull;
    const int sh = (int)(q & 3) * 8;
    uint32_t v[17];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __ldg(reinterpret_cast<const uint32_t *>(data + q4) + j);
    v[16] = sh ? word_at(data, q4 + 64, total) : 0u;
#pragma unroll
    for (int j = 0; j < 16; ++j) w[j] = bswap(__funnelshift_r(v[j], v[j + 1], sh));
    return;
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) w[j] = 0;
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    const uint64_t pos = off + j;
    const uint32_t byte = pos < len ? data[a + pos] : (pos == len ? 0x80u : 0u);
    w[j >> 2] |= byte << (24 - 8 * (j & 3));
  }
  if (off + 64 == padded) {
    const uint64_t bits = len * 8;
    w[14] = (uint32_t)(bits >> 32);
    w[15] = (uint32_t)bits;
  }
}

// Pass 2: every thread hashes the chunks t, t + G, t + 2G, ... (G threads in
// the grid), one 64-byte block per iteration, so that a lane that finishes a
// chunk goes on with its next one while the rest of its warp is still
// hashing: with about ten chunks per thread the per-lane totals even out.
__global__ void __launch_bounds__(128)
sha256_chunks_kernel(const uint8_t *data, uint64_t total, uint64_t ncuts,
                     uint32_t *digests, uint32_t *sizes) {
  const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t a = 0, len = 0, off = 0, padded = 0;
  uint32_t h[8];
  auto start = [&](uint64_t k) {
    const ulonglong2 r = reinterpret_cast<const ulonglong2 *>(digests)[2 * k];
    a = r.x;
    len = r.y - r.x;
    off = 0;
    padded = ((len + 8) / 64 + 1) * 64;
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = c_H0[j];
  };
  if (i < ncuts) start(i);
  while (i < ncuts) {
    uint32_t w[16];
    message_block(data, total, a, len, off, padded, w);
    compress(h, w);
    off += 64;
    if (off == padded) {
      uint32_t *out = digests + i * 8;
#pragma unroll
      for (int j = 0; j < 8; ++j) out[j] = bswap(h[j]);  // bytes in digest order
      if (sizes) sizes[i] = (uint32_t)len;
      i += G;
      if (i < ncuts) start(i);
    }
  }
}

// Insert every chunk's fingerprint into an open-addressing table of chunk
// indices (linear probing, full 32-byte comparison); the first chunk with a
// fingerprint counts as distinct.  out[0] += distinct chunks, out[1] +=
// their bytes.
__global__ void dedup_insert_kernel(const uint32_t *digests, const uint32_t *sizes,
                                    uint64_t n, uint32_t *table, uint64_t mask,
                                    unsigned long long *out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t d[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) d[j] = digests[i * 8 + j];
    uint64_t slot = (((uint64_t)d[1] << 32) | d[0]) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
      const uint32_t prev = atomicCAS(&table[slot], kEmpty, (uint32_t)i);
      if (prev == kEmpty) {
        atomicAdd(&out[0], 1ull);
        atomicAdd(&out[1], (unsigned long long)sizes[i]);
        break;
      }
      bool same = true;
#pragma unroll
      for (int j = 0; j < 8; ++j) same &= digests[(uint64_t)prev * 8 + j] == d[j];
      if (same) break;
      slot = (slot + 1) & mask;
    }
  }
}

uint64_t table_slots(uint64_t nchunks) {
  uint64_t s = 1024;
  while (s < 2 * nchunks) s <<= 1;
  return s;
}

}  // namespace

extern "C" {

int seqcdc_fingerprint_batch(const uint8_t *d_data, uint64_t total_bytes,
                             const uint64_t *d_offsets, uint64_t nfiles,
                             const uint64_t *d_cuts, const uint64_t *d_cut_offsets,
                             uint64_t ncuts, uint8_t *d_digests, uint32_t *d_sizes,
                             void *stream) {
  if (ncuts == 0) return SEQCDC_OK;
  if (!d_data || !d_offsets || !d_cuts || !d_cut_offsets || !d_digests || nfiles == 0)
    return SEQCDC_EINVAL;
  if (((uintptr_t)d_data & 15u) || ((uintptr_t)d_digests & 3u) || ((uintptr_t)d_sizes & 3u))
    return SEQCDC_EINVAL;
  if (ncuts >= 0xffffffffull) return SEQCDC_ERANGE;
  if (!constants_ready()) return SEQCDC_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t *dig = reinterpret_cast<uint32_t *>(d_digests);
  const uint64_t blocks = (ncuts + 255) / 256;
  chunk_ranges_kernel<<<(unsigned)(blocks < 65535u * 8 ? blocks : 65535u * 8), 256, 0, st>>>(
      d_offsets, nfiles, d_cuts, d_cut_offsets, ncuts, dig);
  // Persistent grid: as many 128-thread blocks as are resident at once.
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sha256_chunks_kernel, 128, 0) !=
          cudaSuccess)
    return SEQCDC_ECUDA;
  uint64_t grid = (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
  const uint64_t need = (ncuts + 127) / 128;
  if (grid > need) grid = need;
  sha256_chunks_kernel<<<(unsigned)grid, 128, 0, st>>>(d_data, total_bytes, ncuts, dig, d_sizes);
  return cudaGetLastError() == cudaSuccess ? SEQCDC_OK : SEQCDC_ECUDA;
}

size_t seqcdc_dedup_table_bytes(uint64_t nchunks) {
  return (size_t)table_slots(nchunks) * sizeof(uint32_t);
}

int seqcdc_dedup(const uint8_t *d_digests, const uint32_t *d_sizes, uint64_t nchunks,
                 void *d_table, size_t table_bytes, uint64_t *d_out, void *stream) {
  if (!d_out) return SEQCDC_EINVAL;
  if (nchunks && (!d_digests || !d_sizes || !d_table)) return SEQCDC_EINVAL;
  if (((uintptr_t)d_digests & 3u) || ((uintptr_t)d_table & 3u) || ((uintptr_t)d_out & 7u))
    return SEQCDC_EINVAL;
  if (nchunks >= 0xffffffffull) return SEQCDC_ERANGE;
  const uint64_t slots = table_slots(nchunks);
  if (table_bytes < slots * sizeof(uint32_t)) return SEQCDC_ECAPACITY;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(d_out, 0, 2 * sizeof(uint64_t), st) != cudaSuccess) return SEQCDC_ECUDA;
  if (nchunks == 0) return SEQCDC_OK;
  if (cudaMemsetAsync(d_table, 0xff, slots * sizeof(uint32_t), st) != cudaSuccess)
    return SEQCDC_ECUDA;
  const uint64_t blocks = (nchunks + 255) / 256;
  dedup_insert_kernel<<<(unsigned)(blocks < 65535u * 8 ? blocks : 65535u * 8), 256, 0, st>>>(
      reinterpret_cast<const uint32_t *>(d_digests), d_sizes, nchunks,
      static_cast<uint32_t *>(d_table), slots - 1,
      reinterpret_cast<unsigned long long *>(d_out));
  return cudaGetLastError() == cudaSuccess ? SEQCDC_OK : SEQCDC_ECUDA;
}

}  // extern "C"
