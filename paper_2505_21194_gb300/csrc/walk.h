// walk.h -- internal interface of the chain-walking path (walk.cu), called
// by the C entry points in seqcdc.cu.  Not part of the public ABI.
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "seqcdc.h"

namespace seqcdc_walk {

// Piece size a call runs with: `piece_bytes` from the tuning (0 = default:
// 768 KiB, or 384 x min_size when min_size exceeds 4 KiB), rounded up to
// 64 KiB, at least 4 x max_size, at most 64 MiB.
uint32_t pick_piece(const seqcdc_params_t *p, const seqcdc_tuning_t *t);

// Workspace bytes of one call over `total` bytes in `nfiles` files.
size_t workspace_bytes(const seqcdc_params_t *p, uint64_t total, uint64_t nfiles,
                       uint32_t piece);

// One chunking call (arguments as seqcdc_chunk / seqcdc_chunk_batch; the
// parameters are already validated).  `host_data`: d_data is pinned host
// memory mapped into the device's address space (read in place).
// `prof_begin` / `prof_end` (may be null) are recorded around the piece-walk
// kernel.
int run(const seqcdc_params_t *p, const uint8_t *d_data, uint64_t total,
        const uint64_t *d_offsets, uint64_t nfiles, uint64_t *d_cuts, uint64_t cap,
        uint64_t *d_cut_offsets, uint64_t *d_count, void *d_ws, size_t ws_bytes,
        uint32_t piece, int sms, bool host_data, void *stream, void *prof_begin,
        void *prof_end);

}  // namespace seqcdc_walk
